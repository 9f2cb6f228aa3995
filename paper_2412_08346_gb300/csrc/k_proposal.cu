// Learned initial-pose proposal (the data-driven initialisation the paper names
// as future work, after its Section VII ablation on mixture-of-Gaussian
// initialisations): PointNet-style encoder of the object cloud -> per-preshape
// mixture of SE(3) densities; forward, mixture loss, backward, Adam and
// sampling kernels.  Weights and stored activations are bfloat16 (round to
// nearest even), every product is accumulated in float32; master weights,
// gradients and the Adam state are float32.  The two per-point bfloat16
// contractions of the encoder (layers 2 and 3, every point of every cloud) run on
// the tensor cores (tcgen05, kind::f16); the head layers (one row per object) and
// the backward pass (float32 gradients as operands, which a bfloat16 or tf32 MMA
// would round) run as float32 SIMT GEMMs.
//
// Network (x_i = r_i - centroid; W row-major [out][in]):
//   h1 = relu(W1 x + b1) 3->64, h2 = relu(W2 h1 + b2) 64->128,
//   h3 = relu(W3 h2 + b3) 128->256, g = max over points (ties: lowest point),
//   z = relu(W4 g + b4) 256->256, o = W5 z + b5 256->P*16*10.
// Mixture per preshape p, component c (raw o[0..9]): pi = softmax(o0),
// mu = 0.1 (o1, o2, o3), sigma = 0.1 exp(clip(o4, -4, 1)), nu = (o5..o8)/|.|,
// kappa = 4 exp(clip(o9, -2, 3)); log p(t, q) = LSE_c[log pi_c - |t' - mu_c|^2 /
// (2 sigma_c^2) - 3 log sigma_c + kappa_c (nu_c.q)^2 - log M(1/2, 2, kappa_c)]
// - 1.5 log 2 pi - log 2 pi^2: a Gaussian in translation times a Watson density on
// the quaternion sphere (q and -q score alike; M = Kummer's 1F1, summed as its
// series).  Loss of one object: -(1 / (P T)) sum over preshapes and targets.
//
// Backward: the per-object gradients are written to per-object slices and
// summed in object order, so a training step is deterministic.
#include "../../include/asicp_proposal.h"
#include "asicp_internal.cuh"
#include "tcgen05.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace asicp {
namespace {

typedef __nv_bfloat16 bf16;
constexpr int kC = ASICP_PROP_COMPONENTS, kRaw = ASICP_PROP_RAW;
constexpr int kH1 = 64, kH2 = 128, kH3 = 256, kHead = 256;
constexpr int kMaxPre = 16, kMaxPoints = 65536, kMaxBatch = 256;

struct Layer {
    int out, in;
    size_t w, b;   // offsets of W and b in the flat parameters
};

void layers_for(int P, Layer L[5])
{
    const int dims[5][2] = {{kH1, 3}, {kH2, kH1}, {kH3, kH2}, {kHead, kH3}, {P * kC * kRaw, kHead}};
    size_t off = 0;
    for (int l = 0; l < 5; ++l) {
        L[l].out = dims[l][0];
        L[l].in = dims[l][1];
        L[l].w = off;
        off += (size_t)L[l].out * L[l].in;
        L[l].b = off;
        off += L[l].out;
    }
}

size_t params_for(int P)
{
    Layer L[5];
    layers_for(P, L);
    return L[4].b + L[4].out;
}

__device__ __forceinline__ float ldf(const float *p, long long i) { return p[i]; }
__device__ __forceinline__ float ldf(const bf16 *p, long long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void stf(float *p, long long i, float v) { p[i] = v; }
__device__ __forceinline__ void stf(bf16 *p, long long i, float v) { p[i] = __float2bfloat16_rn(v); }

// ---------------------------------------------------------------- batched GEMM
// C[z][m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) (relu) (* (mask[m][n] > 0)),
// A(m, k) = AT ? A[k lda + m] : A[m lda + k], B(k, n) = BT ? B[n ldb + k] : B[k ldb + n];
// z = blockIdx.z with element strides sA, sB, sC, sM.  64 x 64 tiles, k-steps of 16.
struct GemmArgs {
    const void *A, *B;
    void *C;
    const float *bias;
    const bf16 *mask;
    int M, N, K, lda, ldb, ldc, ldm;
    long long sA, sB, sC, sM;
    int relu;
};

constexpr int kTM = 64, kTN = 64, kTK = 16, kGemmThreads = 256;

template <typename TA, typename TB, typename TC, bool AT, bool BT>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(const GemmArgs g)
{
    __shared__ float As[kTK][kTM + 4];
    __shared__ float Bs[kTK][kTN + 4];
    const TA *A = static_cast<const TA *>(g.A) + (long long)blockIdx.z * g.sA;
    const TB *B = static_cast<const TB *>(g.B) + (long long)blockIdx.z * g.sB;
    TC *C = static_cast<TC *>(g.C) + (long long)blockIdx.z * g.sC;
    const bf16 *mask = g.mask ? g.mask + (long long)blockIdx.z * g.sM : nullptr;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += kTK) {
#pragma unroll
        for (int r = 0; r < (kTM * kTK) / kGemmThreads; ++r) {
            const int e = tid + r * kGemmThreads;
            const int mm = AT ? e % kTM : e / kTK, kk = AT ? e / kTM : e % kTK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < g.M && k < g.K) ? ldf(A, AT ? (long long)k * g.lda + m : (long long)m * g.lda + k) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < (kTN * kTK) / kGemmThreads; ++r) {
            const int e = tid + r * kGemmThreads;
            const int nn = BT ? e / kTK : e % kTN, kk = BT ? e % kTK : e / kTN;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < g.N && k < g.K) ? ldf(B, BT ? (long long)n * g.ldb + k : (long long)k * g.ldb + n) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (g.bias) v += g.bias[n];
            if (g.relu) v = fmaxf(v, 0.f);
            if (mask && !(__bfloat162float(mask[(long long)m * g.ldm + n]) > 0.f)) v = 0.f;
            stf(C, (long long)m * g.ldc + n, v);
        }
    }
}

template <typename TA, typename TB, typename TC, bool AT, bool BT>
cudaError_t gemm(const GemmArgs &g, int batch, cudaStream_t st)
{
    const dim3 grid((g.N + kTN - 1) / kTN, (g.M + kTM - 1) / kTM, batch);
    gemm_kernel<TA, TB, TC, AT, BT><<<grid, kGemmThreads, 0, st>>>(g);
    return cudaGetLastError();
}

GemmArgs gargs(const void *A, int lda, const void *B, int ldb, void *C, int ldc, int M, int N, int K)
{
    GemmArgs g{};
    g.A = A; g.B = B; g.C = C;
    g.lda = lda; g.ldb = ldb; g.ldc = ldc;
    g.M = M; g.N = N; g.K = K;
    return g;
}

// ---------------------------------------------------------------- encoder layers on the tensor cores
// C[r][n] = bf16(relu(sum_k A[r][k] W[n][k] + bias[n])) for the per-point layers 2
// and 3 (K = 64 -> N = 128, K = 128 -> N = 256), both operands bfloat16: one CTA per
// 128 points, the 128 x K rows and the whole N x K weight matrix staged in shared
// memory in the no-swizzle K-major layout, K / 16 tcgen05 MMAs (kind::f16, bf16
// operands, float32 accumulation in tensor memory) issued by one thread, then
// each warp reads its 32 rows back 32 columns at a time, adds the bias, applies
// the ReLU and rounds to bfloat16.  Products of bfloat16 values are exact in
// float32, as in the SIMT kernel; the order of the float32 additions differs.  The
// wait for the MMAs is bounded: on expiry the CTA sets *err and writes nothing.
template <int K, int N>
__global__ void __launch_bounds__(128) dense_relu_tc_kernel(const bf16 *A, const bf16 *W, const float *bias, bf16 *C,
                                                            long long rows, int *err)
{
    constexpr unsigned kLbo = 128, kSbo = K * 16;     // K-adjacent core matrices; 8-row groups
    constexpr unsigned kABytes = 128u * K * 2u;
    constexpr uint32_t kIdesc = tc_idesc_f16(true, N, 128);
    static_assert(K % 16 == 0 && N % 32 == 0 && N >= 32 && N <= 256 && (N & (N - 1)) == 0, "layer shape");
    extern __shared__ __align__(1024) unsigned char sm_dense[];
    unsigned char *sA = sm_dense, *sW = sm_dense + kABytes;
    __shared__ __align__(8) unsigned long long done;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long r = (long long)blockIdx.x * 128 + tid;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(A + r * K);
#pragma unroll
        for (int j = 0; j < K / 8; ++j) {
            const uint4 v = r < rows ? src[j] : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sA + kmajor_offset(tid, 8 * j, kLbo, kSbo)) = v;
        }
        for (int n = tid; n < N; n += 128) {
            const uint4 *ws = reinterpret_cast<const uint4 *>(W + (size_t)n * K);
#pragma unroll
            for (int j = 0; j < K / 8; ++j) *reinterpret_cast<uint4 *>(sW + kmajor_offset(n, 8 * j, kLbo, kSbo)) = ws[j];
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc_alloc(&s_tmem, N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        const unsigned a0 = smem_u32(sA), w0 = smem_u32(sW);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk)
            tc_mma_f16(tmem, tc_smem_desc(a0 + kk * 2 * kLbo, kLbo, kSbo), tc_smem_desc(w0 + kk * 2 * kLbo, kLbo, kSbo),
                       kIdesc, (uint32_t)kk);
        tc_commit(&done);
    }
    bool ok = mbar_wait_warp(&done, 0);
    if (!ok && (tid & 31) == 0) atomicExch(err, kDevTimeout);
    tc_fence_after();
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (ok && r < rows) {
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const bf16 lo = __float2bfloat16_rn(fmaxf(v[2 * i] + bias[c0 + 2 * i], 0.f));
                const bf16 hi = __float2bfloat16_rn(fmaxf(v[2 * i + 1] + bias[c0 + 2 * i + 1], 0.f));
                w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(C + r * N + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
    }
    if (!ok) mbar_wait_warp(&done, 0);   // the MMAs must be done before the columns are freed (bounded)
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, N);
    }
}

// Shared memory of a CTA: its operands, and at least enough that no more CTAs fit on
// an SM than its 512 tensor-memory columns hold (an allocation beyond them would
// wait for another CTA to finish).
template <int K, int N>
constexpr size_t dense_smem_bytes()
{
    constexpr size_t operands = 128u * K * 2u + (size_t)N * K * 2u;
    constexpr size_t per_sm = 228u * 1024u, floor_ = per_sm / (512 / N + 1) + 1024u;
    return operands > floor_ ? operands : floor_;
}

template <int K, int N>
cudaError_t launch_dense_relu_tc(const bf16 *A, const bf16 *W, const float *bias, bf16 *C, long long rows, int *err,
                                 cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(dense_relu_tc_kernel<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dense_smem_bytes<K, N>());
    if (e != cudaSuccess) return e;
    dense_relu_tc_kernel<K, N><<<(unsigned)((rows + 127) / 128), 128, dense_smem_bytes<K, N>(), st>>>(A, W, bias, C,
                                                                                                     rows, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small kernels
// centroid (float64) and the centred input x [B][npts][4] in bfloat16 (4th lane 0)
__global__ void center_kernel(const float *clouds, int npts, float *cen, bf16 *x)
{
    __shared__ double red[3][32];
    const int b = blockIdx.x;
    const float *r = clouds + (size_t)b * npts * 3;
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < npts; i += blockDim.x)
        for (int c = 0; c < 3; ++c) s[c] += (double)r[(size_t)i * 3 + c];
    for (int c = 0; c < 3; ++c) {
        double v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    __shared__ double mean[3];
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        mean[threadIdx.x] = v / npts;
        if (cen) cen[b * 3 + threadIdx.x] = (float)mean[threadIdx.x];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        bf16 *xo = x + ((size_t)b * npts + i) * 4;
        for (int c = 0; c < 3; ++c) xo[c] = __float2bfloat16_rn((float)((double)r[(size_t)i * 3 + c] - mean[c]));
        xo[3] = __float2bfloat16_rn(0.f);
    }
}

// h1 = relu(W1 x + b1) for every point (one thread per point and channel)
__global__ void layer1_kernel(const bf16 *x, const bf16 *W1, const float *b1, bf16 *h1, long long rows)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= rows * kH1) return;
    const long long r = e / kH1;
    const int c = (int)(e - r * kH1);
    const bf16 *xr = x + r * 4;
    float v = b1[c];
    for (int k = 0; k < 3; ++k) v = fmaf(__bfloat162float(W1[c * 3 + k]), __bfloat162float(xr[k]), v);
    h1[e] = __float2bfloat16_rn(fmaxf(v, 0.f));
}

// g = max over points of h3 per channel, with the lowest maximising point
__global__ void maxpool_kernel(const bf16 *h3, int npts, bf16 *g, int *arg)
{
    const int b = blockIdx.x, ch = threadIdx.x;
    const bf16 *hb = h3 + (size_t)b * npts * kH3;
    float best = -1.f;
    int bi = 0;
    for (int i = 0; i < npts; ++i) {
        const float v = __bfloat162float(hb[(size_t)i * kH3 + ch]);
        if (v > best) { best = v; bi = i; }
    }
    g[b * kH3 + ch] = __float2bfloat16_rn(best);
    arg[b * kH3 + ch] = bi;
}

struct Mix {
    float logpi[kC], mu[kC][3], sigma[kC], nu[kC][4], nv[kC], kappa[kC], logm[kC], dlogm[kC];
    int inside[kC], kin[kC];
};

// Kummer's 1F1(a; b; k) by its series (k <= 80 here: under 200 terms)
__device__ double kummer(double a, double b, double k)
{
    double t = 1.0, s = 1.0;
    for (int n = 0; n < 400; ++n) {
        t *= (a + n) / (b + n) * k / (n + 1);
        s += t;
        if (t < 1e-17 * s) break;
    }
    return s;
}

// Mixture parameters of one preshape from its raw outputs; thread c < kC fills
// component c (call with at least kC threads, then synchronise).
__device__ void mixture_params(const float *o, Mix &m, int c)
{
    if (c >= kC) return;
    float amax = -INFINITY;
    for (int e = 0; e < kC; ++e) amax = fmaxf(amax, o[e * kRaw]);
    float se = 0.f;
    for (int e = 0; e < kC; ++e) se += expf(o[e * kRaw] - amax);
    const float *oc = o + c * kRaw;
    m.logpi[c] = oc[0] - (amax + logf(se));
    for (int k = 0; k < 3; ++k) m.mu[c][k] = 0.1f * oc[1 + k];
    m.inside[c] = oc[4] > -4.f && oc[4] < 1.f;
    m.sigma[c] = 0.1f * expf(fminf(fmaxf(oc[4], -4.f), 1.f));
    const float n = fmaxf(sqrtf(oc[5] * oc[5] + oc[6] * oc[6] + oc[7] * oc[7] + oc[8] * oc[8]), 1e-6f);
    m.nv[c] = n;
    for (int k = 0; k < 4; ++k) m.nu[c][k] = oc[5 + k] / n;
    m.kin[c] = oc[9] > -2.f && oc[9] < 3.f;
    const float kap = 4.f * expf(fminf(fmaxf(oc[9], -2.f), 3.f));
    m.kappa[c] = kap;
    const double m0 = kummer(0.5, 2.0, kap), m1 = kummer(1.5, 3.0, kap);
    m.logm[c] = (float)log(m0);
    m.dlogm[c] = (float)(0.25 * m1 / m0);
}

// Loss of preshape p of object b and its gradient with respect to the raw outputs.
// One CTA per (p, b), thread j = target j; per component the contributions are
// summed by warp shuffles and then over warps in warp order (deterministic).
constexpr int kLossThreads = ASICP_PROP_MAX_TARGETS;

__global__ void __launch_bounds__(kLossThreads) loss_kernel(const float *out, const float *cen, const float *targets,
                                                            int P, int T, float *dO, float *lossp)
{
    __shared__ Mix mx;
    __shared__ float part[kLossThreads / 32][kC][kRaw];
    __shared__ float lpart[kLossThreads / 32];
    const int p = blockIdx.x, b = blockIdx.y, j = threadIdx.x, lane = j & 31, warp = j >> 5;
    const float *o = out + ((size_t)b * P + p) * kC * kRaw;
    mixture_params(o, mx, j);
    __syncthreads();
    const bool live = j < T;
    float t[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f};
    if (live) {
        const float *tg = targets + (((size_t)b * P + p) * T + j) * 7;
        for (int k = 0; k < 3; ++k) t[k] = tg[k] - cen[b * 3 + k];
        for (int k = 0; k < 4; ++k) q[k] = tg[3 + k];
    }
    float ell[kC], dot[kC], d2[kC];
    float emax = -INFINITY;
    for (int c = 0; c < kC; ++c) {
        float dd = 0.f;
        for (int k = 0; k < 3; ++k) { const float e = t[k] - mx.mu[c][k]; dd = fmaf(e, e, dd); }
        float dq = 0.f;
        for (int k = 0; k < 4; ++k) dq = fmaf(q[k], mx.nu[c][k], dq);
        d2[c] = dd;
        dot[c] = dq;
        const float s = mx.sigma[c];
        ell[c] = mx.logpi[c] - dd / (2.f * s * s) - 3.f * logf(s) + mx.kappa[c] * dq * dq - mx.logm[c];
        emax = fmaxf(emax, ell[c]);
    }
    float se = 0.f;
    for (int c = 0; c < kC; ++c) se += expf(ell[c] - emax);
    const float lse = emax + logf(se);
    // constant: -1.5 log(2 pi) - log(2 pi^2)
    float nll = live ? -(lse - 2.75681559961402f - 2.98260695225875f) : 0.f;
    const float w = -1.f / (float)(P * T);
    for (int c = 0; c < kC; ++c) {
        const float r = live ? expf(ell[c] - lse) : 0.f;
        const float s = mx.sigma[c];
        float v[kRaw];
        v[0] = live ? w * (r - expf(mx.logpi[c])) : 0.f;
        for (int k = 0; k < 3; ++k) v[1 + k] = w * 0.1f * r * (t[k] - mx.mu[c][k]) / (s * s);
        v[4] = mx.inside[c] ? w * r * (d2[c] / (s * s * s) - 3.f / s) * s : 0.f;
        float dn[4], pr = 0.f;
        for (int k = 0; k < 4; ++k) { dn[k] = r * 2.f * mx.kappa[c] * dot[c] * q[k]; pr = fmaf(dn[k], mx.nu[c][k], pr); }
        for (int k = 0; k < 4; ++k) v[5 + k] = w * (dn[k] - pr * mx.nu[c][k]) / mx.nv[c];
        v[9] = mx.kin[c] ? w * r * (dot[c] * dot[c] - mx.dlogm[c]) * mx.kappa[c] : 0.f;
        for (int k = 0; k < kRaw; ++k) {
            float x = v[k];
            for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o2);
            if (lane == 0) part[warp][c][k] = x;
        }
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) nll += __shfl_xor_sync(0xffffffffu, nll, o2);
    if (lane == 0) lpart[warp] = nll;
    __syncthreads();
    for (int e = j; e < kC * kRaw; e += blockDim.x) {
        const int c = e / kRaw, k = e % kRaw;
        float s = 0.f;
        for (int wv = 0; wv < kLossThreads / 32; ++wv) s += part[wv][c][k];
        dO[((size_t)b * P + p) * kC * kRaw + e] = s;
    }
    if (j == 0) {
        float s = 0.f;
        for (int wv = 0; wv < kLossThreads / 32; ++wv) s += lpart[wv];
        lossp[b * P + p] = s;
    }
}

// dh3 (zeroed beforehand): the max-pool routes dg to the maximising point, through the relu
__global__ void scatter_dh3_kernel(const float *dg, const int *arg, const bf16 *h3, int npts, float *dh3)
{
    const int b = blockIdx.x, ch = threadIdx.x;
    const int i = arg[b * kH3 + ch];
    const size_t e = ((size_t)b * npts + i) * kH3 + ch;
    dh3[e] = __bfloat162float(h3[e]) > 0.f ? dg[b * kH3 + ch] : 0.f;
}

// out[z][c] = sum over rows of D[z][row][c] (bias gradients), rows in order
__global__ void colsum_kernel(const float *D, int rows, int cols, long long sD, float *out, long long sOut)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y;
    if (c >= cols) return;
    const float *d = D + z * sD;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += d[(size_t)r * cols + c];
    out[z * sOut + c] = s;
}

// grad[j] = (1/B) sum_b slices[b][j], objects in order
__global__ void reduce_slices_kernel(const float *slices, int B, size_t np, float *grad)
{
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += slices[(size_t)b * np + j];
    grad[j] = s / (float)B;
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, size_t n, float lr, float bc1, float bc2)
{
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float gj = g[j];
    const float mj = 0.9f * m[j] + 0.1f * gj;
    const float vj = 0.999f * v[j] + 0.001f * gj * gj;
    m[j] = mj;
    v[j] = vj;
    w[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + 1e-8f);
}

__global__ void to_bf16_kernel(const float *src, bf16 *dst, size_t n)
{
    const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j < n) dst[j] = __float2bfloat16_rn(src[j]);
}

// theta [B][P][K][7] from the mixtures and the caller's draws [B][P][K][8]
__global__ void sample_kernel(const float *out, const float *cen, const float *draws, int B, int P, int K,
                              float *theta)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)B * P * K) return;
    const int b = (int)(e / ((long long)P * K)), p = (int)((e / K) % P);
    const float *o = out + ((size_t)b * P + p) * kC * kRaw;
    const float *d = draws + e * 8;
    float amax = -INFINITY;
    for (int c = 0; c < kC; ++c) amax = fmaxf(amax, o[c * kRaw]);
    float cdf[kC], tot = 0.f;
    for (int c = 0; c < kC; ++c) { tot += expf(o[c * kRaw] - amax); cdf[c] = tot; }
    const float u = d[0] * tot;
    int c = kC - 1;
    for (int k = kC - 1; k >= 0; --k)
        if (cdf[k] > u) c = k;
    const float *oc = o + c * kRaw;
    const float sigma = 0.1f * expf(fminf(fmaxf(oc[4], -4.f), 1.f));
    float *th = theta + e * 7;
    for (int k = 0; k < 3; ++k) th[k] = cen[b * 3 + k] + 0.1f * oc[1 + k] + sigma * d[1 + k];
    const float n = fmaxf(sqrtf(oc[5] * oc[5] + oc[6] * oc[6] + oc[7] * oc[7] + oc[8] * oc[8]), 1e-6f);
    const float kap = 4.f * expf(fminf(fmaxf(oc[9], -2.f), 3.f));
    const float spread = rsqrtf(2.f * kap);
    float qv[4], qq = 0.f;
    for (int k = 0; k < 4; ++k) { qv[k] = oc[5 + k] / n + d[4 + k] * spread; qq = fmaf(qv[k], qv[k], qq); }
    const float inv = 1.f / sqrtf(qq);
    for (int k = 0; k < 4; ++k) th[3 + k] = qv[k] * inv;
}

// ---------------------------------------------------------------- handle
struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct PropErr {
    asicp_status st;
};

void pck(cudaError_t e)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw PropErr{e == cudaErrorMemoryAllocation ? ASICP_ERR_OOM : ASICP_ERR_CUDA};
    }
}

void alloc(Buf &b, size_t bytes) { pck(cudaMalloc(&b.p, bytes < 16 ? 16 : bytes)); }

}  // namespace
}  // namespace asicp

using namespace asicp;

struct asicp_prop {
    int P = 0, npts = 0, maxB = 0, nout = 0;
    size_t np = 0;
    Layer L[5];
    cudaStream_t st = nullptr;
    long long step = 0;
    int lastB = 0;
    Buf w, m, v, grad, slices, wbf, clouds, tg, cen, x, h1, h2, h3, g, arg, z, o, dO, lossp, dz, dg, dh3, dh2, dh1,
        outb, drawb, thetab, errw;
};

namespace {

template <class F>
asicp_status prop_guard(F &&f)
{
    try {
        f();
        return ASICP_OK;
    } catch (const PropErr &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        return ASICP_ERR_OOM;
    }
}

// After a synchronisation: a bounded device wait that expired (the tensor-core
// layers) is reported as TIMEOUT, once.
void check_device_error(asicp_prop *pr)
{
    int e = 0;
    pck(cudaMemcpy(&e, pr->errw.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != kDevOk) {
        pck(cudaMemset(pr->errw.p, 0, sizeof(int)));
        throw PropErr{ASICP_ERR_TIMEOUT};
    }
}

// device copy of an input that may be host memory
const float *staged(asicp_prop *pr, const float *src, size_t n, Buf &buf)
{
    pck(cudaMemcpyAsync(buf.p, src, n * sizeof(float), cudaMemcpyDefault, pr->st));
    return buf.as<float>();
}

void forward_impl(asicp_prop *pr, const float *clouds_dev, int B)
{
    cudaStream_t st = pr->st;
    const long long rows = (long long)B * pr->npts;
    const bf16 *W = pr->wbf.as<bf16>();
    const float *wf = pr->w.as<float>();
    center_kernel<<<B, 256, 0, st>>>(clouds_dev, pr->npts, pr->cen.as<float>(), pr->x.as<bf16>());
    pck(cudaGetLastError());
    layer1_kernel<<<(unsigned)((rows * kH1 + 255) / 256), 256, 0, st>>>(pr->x.as<bf16>(), W + pr->L[0].w,
                                                                        wf + pr->L[0].b, pr->h1.as<bf16>(), rows);
    pck(cudaGetLastError());
    // layers 2 and 3: bfloat16 contractions over every point, on the tensor cores
    pck(launch_dense_relu_tc<kH1, kH2>(pr->h1.as<bf16>(), W + pr->L[1].w, wf + pr->L[1].b, pr->h2.as<bf16>(), rows,
                                        pr->errw.as<int>(), st));
    pck(launch_dense_relu_tc<kH2, kH3>(pr->h2.as<bf16>(), W + pr->L[2].w, wf + pr->L[2].b, pr->h3.as<bf16>(), rows,
                                        pr->errw.as<int>(), st));
    maxpool_kernel<<<B, kH3, 0, st>>>(pr->h3.as<bf16>(), pr->npts, pr->g.as<bf16>(), pr->arg.as<int>());
    pck(cudaGetLastError());
    GemmArgs g4 = gargs(pr->g.p, kH3, W + pr->L[3].w, kH3, pr->z.p, kHead, B, kHead, kH3);
    g4.bias = wf + pr->L[3].b;
    g4.relu = 1;
    pck(gemm<bf16, bf16, bf16, false, true>(g4, 1, st));
    GemmArgs g5 = gargs(pr->z.p, kHead, W + pr->L[4].w, kHead, pr->o.p, pr->nout, B, pr->nout, kHead);
    g5.bias = wf + pr->L[4].b;
    pck(gemm<bf16, bf16, float, false, true>(g5, 1, st));
}

void backward_impl(asicp_prop *pr, int B)
{
    cudaStream_t st = pr->st;
    const int n = pr->npts, no = pr->nout;
    const long long rows = (long long)B * n;
    const bf16 *W = pr->wbf.as<bf16>();
    float *S = pr->slices.as<float>();
    const long long np = (long long)pr->np;
    // head: dW5_b = dO_b (x) z_b, db5_b = dO_b, dz = (dO W5) * (z > 0)
    GemmArgs a = gargs(pr->dO.p, 1, pr->z.p, kHead, S + pr->L[4].w, kHead, no, kHead, 1);
    a.sA = no; a.sB = kHead; a.sC = np;
    pck(gemm<float, bf16, float, false, false>(a, B, st));
    colsum_kernel<<<dim3((no + 255) / 256, B), 256, 0, st>>>(pr->dO.as<float>(), 1, no, no, S + pr->L[4].b, np);
    pck(cudaGetLastError());
    GemmArgs d = gargs(pr->dO.p, no, W + pr->L[4].w, kHead, pr->dz.p, kHead, B, kHead, no);
    d.mask = pr->z.as<bf16>();
    d.ldm = kHead;
    pck(gemm<float, bf16, float, false, false>(d, 1, st));
    // dW4_b = dz_b (x) g_b, db4_b = dz_b, dg = dz W4
    a = gargs(pr->dz.p, 1, pr->g.p, kH3, S + pr->L[3].w, kH3, kHead, kH3, 1);
    a.sA = kHead; a.sB = kH3; a.sC = np;
    pck(gemm<float, bf16, float, false, false>(a, B, st));
    colsum_kernel<<<dim3(1, B), 256, 0, st>>>(pr->dz.as<float>(), 1, kHead, kHead, S + pr->L[3].b, np);
    pck(cudaGetLastError());
    d = gargs(pr->dz.p, kHead, W + pr->L[3].w, kH3, pr->dg.p, kH3, B, kH3, kHead);
    pck(gemm<float, bf16, float, false, false>(d, 1, st));
    // max-pool and layer 3
    pck(cudaMemsetAsync(pr->dh3.p, 0, sizeof(float) * rows * kH3, st));
    scatter_dh3_kernel<<<B, kH3, 0, st>>>(pr->dg.as<float>(), pr->arg.as<int>(), pr->h3.as<bf16>(), n,
                                          pr->dh3.as<float>());
    pck(cudaGetLastError());
    a = gargs(pr->dh3.p, kH3, pr->h2.p, kH2, S + pr->L[2].w, kH2, kH3, kH2, n);
    a.sA = (long long)n * kH3; a.sB = (long long)n * kH2; a.sC = np;
    pck(gemm<float, bf16, float, true, false>(a, B, st));
    colsum_kernel<<<dim3(1, B), 256, 0, st>>>(pr->dh3.as<float>(), n, kH3, (long long)n * kH3, S + pr->L[2].b, np);
    pck(cudaGetLastError());
    d = gargs(pr->dh3.p, kH3, W + pr->L[2].w, kH2, pr->dh2.p, kH2, (int)rows, kH2, kH3);
    d.mask = pr->h2.as<bf16>();
    d.ldm = kH2;
    pck(gemm<float, bf16, float, false, false>(d, 1, st));
    // layer 2
    a = gargs(pr->dh2.p, kH2, pr->h1.p, kH1, S + pr->L[1].w, kH1, kH2, kH1, n);
    a.sA = (long long)n * kH2; a.sB = (long long)n * kH1; a.sC = np;
    pck(gemm<float, bf16, float, true, false>(a, B, st));
    colsum_kernel<<<dim3(1, B), 256, 0, st>>>(pr->dh2.as<float>(), n, kH2, (long long)n * kH2, S + pr->L[1].b, np);
    pck(cudaGetLastError());
    d = gargs(pr->dh2.p, kH2, W + pr->L[1].w, kH1, pr->dh1.p, kH1, (int)rows, kH1, kH2);
    d.mask = pr->h1.as<bf16>();
    d.ldm = kH1;
    pck(gemm<float, bf16, float, false, false>(d, 1, st));
    // layer 1
    a = gargs(pr->dh1.p, kH1, pr->x.p, 4, S + pr->L[0].w, 3, kH1, 3, n);
    a.sA = (long long)n * kH1; a.sB = (long long)n * 4; a.sC = np;
    pck(gemm<float, bf16, float, true, false>(a, B, st));
    colsum_kernel<<<dim3(1, B), 256, 0, st>>>(pr->dh1.as<float>(), n, kH1, (long long)n * kH1, S + pr->L[0].b, np);
    pck(cudaGetLastError());
    reduce_slices_kernel<<<(unsigned)((pr->np + 255) / 256), 256, 0, st>>>(S, B, pr->np, pr->grad.as<float>());
    pck(cudaGetLastError());
}

void refresh_bf16(asicp_prop *pr)
{
    to_bf16_kernel<<<(unsigned)((pr->np + 255) / 256), 256, 0, pr->st>>>(pr->w.as<float>(), pr->wbf.as<bf16>(), pr->np);
    pck(cudaGetLastError());
}

}  // namespace

extern "C" {

size_t asicp_prop_num_params(int P)
{
    if (P < 1 || P > kMaxPre) return 0;
    return params_for(P);
}

asicp_status asicp_prop_create(int P, int n_points, int max_batch, void *cuda_stream, asicp_prop **out)
{
    if (!out) return ASICP_ERR_INVALID_ARG;
    *out = nullptr;
    if (P < 1 || P > kMaxPre || n_points < 16 || n_points > kMaxPoints || max_batch < 1 || max_batch > kMaxBatch)
        return ASICP_ERR_INVALID_ARG;
    asicp_prop *pr = new (std::nothrow) asicp_prop();
    if (!pr) return ASICP_ERR_OOM;
    pr->P = P;
    pr->npts = n_points;
    pr->maxB = max_batch;
    pr->nout = P * kC * kRaw;
    layers_for(P, pr->L);
    pr->np = params_for(P);
    pr->st = static_cast<cudaStream_t>(cuda_stream);
    const size_t B = max_batch, rows = B * n_points, np = pr->np;
    asicp_status s = prop_guard([&] {
        alloc(pr->w, np * 4); alloc(pr->m, np * 4); alloc(pr->v, np * 4); alloc(pr->grad, np * 4);
        alloc(pr->slices, B * np * 4); alloc(pr->wbf, np * 2);
        alloc(pr->clouds, rows * 3 * 4); alloc(pr->tg, B * P * ASICP_PROP_MAX_TARGETS * 7 * 4);
        alloc(pr->cen, B * 3 * 4); alloc(pr->x, rows * 4 * 2);
        alloc(pr->h1, rows * kH1 * 2); alloc(pr->h2, rows * kH2 * 2); alloc(pr->h3, rows * kH3 * 2);
        alloc(pr->g, B * kH3 * 2); alloc(pr->arg, B * kH3 * 4); alloc(pr->z, B * kHead * 2);
        alloc(pr->o, B * pr->nout * 4); alloc(pr->dO, B * pr->nout * 4); alloc(pr->lossp, B * P * 4);
        alloc(pr->dz, B * kHead * 4); alloc(pr->dg, B * kH3 * 4);
        alloc(pr->dh3, rows * kH3 * 4); alloc(pr->dh2, rows * kH2 * 4); alloc(pr->dh1, rows * kH1 * 4);
        alloc(pr->outb, B * pr->nout * 4);
        alloc(pr->errw, sizeof(int));
        pck(cudaMemsetAsync(pr->errw.p, 0, sizeof(int), pr->st));
        pck(cudaMemsetAsync(pr->w.p, 0, np * 4, pr->st));
        pck(cudaMemsetAsync(pr->m.p, 0, np * 4, pr->st));
        pck(cudaMemsetAsync(pr->v.p, 0, np * 4, pr->st));
        pck(cudaMemsetAsync(pr->grad.p, 0, np * 4, pr->st));
        refresh_bf16(pr);
        pck(cudaStreamSynchronize(pr->st));
    });
    if (s != ASICP_OK) {
        delete pr;
        return s;
    }
    *out = pr;
    return ASICP_OK;
}

asicp_status asicp_prop_destroy(asicp_prop *pr)
{
    if (!pr) return ASICP_ERR_INVALID_ARG;
    cudaStreamSynchronize(pr->st);
    delete pr;
    return ASICP_OK;
}

asicp_status asicp_prop_set_params(asicp_prop *pr, const float *params)
{
    if (!pr || !params) return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        pck(cudaMemcpyAsync(pr->w.p, params, pr->np * 4, cudaMemcpyDefault, pr->st));
        pck(cudaMemsetAsync(pr->m.p, 0, pr->np * 4, pr->st));
        pck(cudaMemsetAsync(pr->v.p, 0, pr->np * 4, pr->st));
        pr->step = 0;
        refresh_bf16(pr);
        pck(cudaStreamSynchronize(pr->st));
    });
}

asicp_status asicp_prop_get_params(asicp_prop *pr, float *params)
{
    if (!pr || !params) return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        pck(cudaMemcpyAsync(params, pr->w.p, pr->np * 4, cudaMemcpyDefault, pr->st));
        pck(cudaStreamSynchronize(pr->st));
    });
}

asicp_status asicp_prop_forward(asicp_prop *pr, const float *clouds, int B, float *out, float *centroids)
{
    if (!pr || !clouds || !out || B < 1 || B > pr->maxB) return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        const float *c = staged(pr, clouds, (size_t)B * pr->npts * 3, pr->clouds);
        forward_impl(pr, c, B);
        pck(cudaMemcpyAsync(out, pr->o.p, (size_t)B * pr->nout * 4, cudaMemcpyDefault, pr->st));
        if (centroids) pck(cudaMemcpyAsync(centroids, pr->cen.p, (size_t)B * 3 * 4, cudaMemcpyDefault, pr->st));
        pck(cudaStreamSynchronize(pr->st));
        check_device_error(pr);
    });
}

asicp_status asicp_prop_loss_grad(asicp_prop *pr, const float *clouds, const float *targets, int B, int T,
                                  float *loss, float *grad)
{
    if (!pr || !clouds || !targets || !loss || B < 1 || B > pr->maxB || T < 1 || T > ASICP_PROP_MAX_TARGETS)
        return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        const float *c = staged(pr, clouds, (size_t)B * pr->npts * 3, pr->clouds);
        const float *t = staged(pr, targets, (size_t)B * pr->P * T * 7, pr->tg);
        forward_impl(pr, c, B);
        loss_kernel<<<dim3(pr->P, B), kLossThreads, 0, pr->st>>>(pr->o.as<float>(), pr->cen.as<float>(), t, pr->P, T,
                                                                 pr->dO.as<float>(), pr->lossp.as<float>());
        pck(cudaGetLastError());
        backward_impl(pr, B);
        std::vector<float> lp((size_t)B * pr->P);
        pck(cudaMemcpyAsync(lp.data(), pr->lossp.p, lp.size() * 4, cudaMemcpyDeviceToHost, pr->st));
        if (grad) pck(cudaMemcpyAsync(grad, pr->grad.p, pr->np * 4, cudaMemcpyDefault, pr->st));
        pck(cudaStreamSynchronize(pr->st));
        check_device_error(pr);
        double s = 0.0;     // mean over objects of (1 / (P T)) sum over preshapes and targets
        for (float x : lp) s += x;
        *loss = (float)(s / ((double)pr->P * T * B));
        pr->lastB = B;
    });
}

asicp_status asicp_prop_adam_step(asicp_prop *pr, float lr)
{
    if (!pr || !(lr > 0.f) || pr->lastB == 0) return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        ++pr->step;
        const float bc1 = 1.f - powf(0.9f, (float)pr->step), bc2 = 1.f - powf(0.999f, (float)pr->step);
        adam_kernel<<<(unsigned)((pr->np + 255) / 256), 256, 0, pr->st>>>(pr->w.as<float>(), pr->m.as<float>(),
                                                                          pr->v.as<float>(), pr->grad.as<float>(),
                                                                          pr->np, lr, bc1, bc2);
        pck(cudaGetLastError());
        refresh_bf16(pr);
        pck(cudaStreamSynchronize(pr->st));
    });
}

asicp_status asicp_prop_sample(asicp_prop *pr, const float *out, const float *centroids, int B, int K,
                               const float *draws, float *theta)
{
    if (!pr || !out || !centroids || !draws || !theta || B < 1 || B > pr->maxB || K < 1 || K > 4096)
        return ASICP_ERR_INVALID_ARG;
    return prop_guard([&] {
        const size_t n = (size_t)B * pr->P * K;
        Buf dr, th, cn;
        alloc(dr, n * 8 * 4);
        alloc(th, n * 7 * 4);
        alloc(cn, (size_t)B * 3 * 4);
        pck(cudaMemcpyAsync(pr->outb.p, out, (size_t)B * pr->nout * 4, cudaMemcpyDefault, pr->st));
        pck(cudaMemcpyAsync(dr.p, draws, n * 8 * 4, cudaMemcpyDefault, pr->st));
        pck(cudaMemcpyAsync(cn.p, centroids, (size_t)B * 3 * 4, cudaMemcpyDefault, pr->st));
        sample_kernel<<<(unsigned)((n + 255) / 256), 256, 0, pr->st>>>(pr->outb.as<float>(), cn.as<float>(),
                                                                      dr.as<float>(), B, pr->P, K, th.as<float>());
        pck(cudaGetLastError());
        pck(cudaMemcpyAsync(theta, th.p, n * 7 * 4, cudaMemcpyDefault, pr->st));
        pck(cudaStreamSynchronize(pr->st));
    });
}

}  // extern "C"
