// Forward matching: transform + brute-force nearest neighbour + per-particle sums.
//
// For particle (p, j) and gripper point i the kernel forms s'_i = R_j s_i + t_j
// (Algorithm 1, "transform the source cloud") and finds the object point with
// the smallest squared distance, ties to the lowest index (Eq. 1).
//
// Search in two stages, exact in the end:
//  1. Screening, in coordinates relative to the object's frame centre c (the
//     centre of its bounding box, so the screening error does not grow with the
//     object's distance from the origin): with b = fl(r - c) and a = fl(s' - c)
//     the kernel evaluates d~(r) = |b|^2 - 2 a.b (= |a - b|^2 - |a|^2, the same
//     ranking as |s' - r|^2 up to the rounding of a and b) as three fused
//     multiply-adds on precomputed (-2b, |b|^2), two object points per packed
//     f32x2 instruction, and keeps per chunk of kChunk points the chunk minimum
//     with a 3-input min.  Per query it tracks the best two chunk minima
//     b1 <= b2 with their chunk ids, and the third-best b3.
//  2. Exact choice.  With u = 2^-24, B = max |b| and A = |a|, the float32
//     evaluation is within u (4.01 B^2 + 6.02 A B) of |b|^2 - 2 a.b (rounding of
//     |b|^2 plus three roundings of the FMA chain, with sum |a_k b_k| <= A B).
//     The rounding of a and b changes |a - b|^2 - |a|^2 against |s' - r|^2 by a
//     term independent of r (which does not change the ranking) plus at most
//     u (2 B^2 + 4 A B), so d~(r) = |s' - r|^2 + const + e(r) with
//     |e(r)| <= delta = u (6.01 B^2 + 10.02 A B).  The true nearest point r*
//     therefore has d~(r*) <= b1 + 2 delta, so every chunk whose minimum exceeds
//     that bound is excluded.  If only chunk c1 (and c2 when b2 <= b1 + 2 delta)
//     can hold r*, their points are re-evaluated with the exact-form distance
//     (dx^2 + dy^2 + dz^2 of s' - r in float32, original coordinates) in index
//     order; if a third chunk could (b3 <= b1 + 2 delta, rare), the warp scans
//     the whole cloud for that query together.  The result is the lowest-index
//     minimum of the exact-form float32 distance among all points that can be
//     nearest.
//
// Object tiles are staged in shared memory by 1D bulk (TMA) copies into two
// buffers guarded by mbarriers; waits are bounded and report a timeout through
// the error word instead of hanging.
//
// The epilogue accumulates, in float64, the sums that the cost and gradient of
// Eqs. 13-17 are linear in: sum r_i (3), sum r_i s_i^T (9), sum |r_i|^2 (1),
// with r_i the matched object point and s_i the untransformed gripper point;
// both are float32, so every product is exact in float64.
#include "asicp_internal.cuh"
#include "async_copy.cuh"

namespace asicp {

namespace {

// Kernel shapes the autotuner chooses from: queries per thread, screening
// chunk, threads per CTA, object points per shared-memory tile (two buffers),
// and the CTAs per SM the register budget is set for.
template <int QPT_, int CHUNK_, int THREADS_, int TILE_, int MINB_>
struct FwdShape {
    static constexpr int QPT = QPT_;
    static constexpr int kChunk = CHUNK_;
    static constexpr int kThreads = THREADS_;
    static constexpr int kTile = TILE_;
    static constexpr int kMinBlocks = MINB_;
    static constexpr int kItem = QPT_ * THREADS_;     // queries per work item at most
    static_assert(kItem <= kFwdItemQueries && kRefTilePts % TILE_ == 0 && TILE_ % CHUNK_ == 0, "shape");
};

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ float min3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

}  // namespace

// One screening + exact pass of the queries [q0, q0 + nq) (nq <= kThreads * Q,
// all on one object) over that object's whole cloud.  Object tiles stream
// through the two shared buffers; `seq` counts the tiles this CTA has consumed,
// which gives each buffer's mbarrier phase.
template <class Shape, int Q>
__device__ __forceinline__ bool match_pass(const FwdArgs &a, const ObjMeta &om, float4 fr, long long q0, int nq,
                                           ulonglong2 *tiles, unsigned long long *full, unsigned long long *never,
                                           int &seq, int *s_abort)
{
    constexpr int kThreads = Shape::kThreads, kChunk = Shape::kChunk, kTile = Shape::kTile;
    const int ntiles = om.Mpad / kTile;
    const unsigned tile_bytes = kTile * 16u;
    if (threadIdx.x == 0) {    // both buffers are free: the previous pass ended with a barrier
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const int b = (seq + t) & 1;
            mbar_arrive_tx(&full[b], tile_bytes);
            bulk_load(tiles + (size_t)b * kTile, om.Rx + (size_t)t * kTile, tile_bytes, &full[b]);
        }
    }
    float sx[Q], sy[Q], sz[Q], win[Q], cm[Q], b1[Q], b2[Q], b3[Q];
    int c1[Q], c2[Q];
    unsigned long long qx[Q], qy[Q], qz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int li = q * kThreads + threadIdx.x;
        float3 o = make_float3(0.f, 0.f, 0.f);
        if (li < nq) {
            const long long g = q0 + li;
            const int pk = (int)(g / a.L.N), i = (int)(g - (long long)pk * a.L.N);
            const int pre = a.L.part_grp[pk] % a.L.P;
            const float *th = a.theta + (size_t)pk * 8;
            float Rm[9];
            quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
            const float4 s = a.S[(size_t)pre * a.L.N + i];
            o = xform_f32(Rm, th[0], th[1], th[2], s.x, s.y, s.z);
        }
        sx[q] = o.x; sy[q] = o.y; sz[q] = o.z;
        // the query relative to the frame centre (a = fl(s' - c))
        const float ax = __fsub_rn(o.x, fr.x), ay = __fsub_rn(o.y, fr.y), az = __fsub_rn(o.z, fr.z);
        qx[q] = pack2(ax, ax); qy[q] = pack2(ay, ay); qz[q] = pack2(az, az);
        const float an = sqrtf(ax * ax + ay * ay + az * az) * 1.001f;
        // 2 delta with a 1 % margin for the float32 evaluation of the bound itself
        win[q] = 2.02f * 5.9604645e-8f * (6.01f * fr.w * fr.w + 10.02f * an * fr.w);
        b1[q] = b2[q] = b3[q] = __int_as_float(0x7f800000);
        c1[q] = c2[q] = 0;
    }

    for (int t = 0; t < ntiles; ++t, ++seq) {
        const int buf = seq & 1;
        // (testing the timeout path: the CTA's first wait is on a barrier nothing arrives at)
        const bool landed = a.expire_test && seq == 0 ? mbar_wait(never, 0u, kTestWaitCycles)
                                                      : mbar_wait(&full[buf], (seq >> 1) & 1);
        if (!landed) {
            atomicExch(a.err, kDevTimeout);
            *s_abort = 1;
        }
        __syncthreads();
        if (*s_abort) return false;
        const ulonglong2 *tp = tiles + (size_t)buf * kTile;
        for (int c = 0; c < kTile / kChunk; ++c) {
#pragma unroll
            for (int q = 0; q < Q; ++q) cm[q] = __int_as_float(0x7f800000);
            const ulonglong2 *cp = tp + c * kChunk;
#pragma unroll 8
            for (int r2 = 0; r2 < kChunk / 2; ++r2) {
                const ulonglong2 A = cp[2 * r2];       // {ax0,ax1} {ay0,ay1}
                const ulonglong2 B = cp[2 * r2 + 1];   // {az0,az1} {w0,w1}
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const unsigned long long d = fma2(qx[q], A.x, fma2(qy[q], A.y, fma2(qz[q], B.x, B.y)));
                    float d0, d1;
                    unpack2(d, d0, d1);
                    cm[q] = min3(cm[q], d0, d1);
                }
            }
            const int gc = t * (kTile / kChunk) + c;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const float v = cm[q];
                const bool n1 = v < b1[q], n2 = v < b2[q];
                b3[q] = n2 ? b2[q] : fminf(b3[q], v);
                b2[q] = n1 ? b1[q] : (n2 ? v : b2[q]);
                c2[q] = n1 ? c1[q] : (n2 ? gc : c2[q]);
                b1[q] = n1 ? v : b1[q];
                c1[q] = n1 ? gc : c1[q];
            }
        }
        __syncthreads();   // every thread is done with this buffer
        if (threadIdx.x == 0 && t + 2 < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_tx(&full[buf], tile_bytes);
            bulk_load(tiles + (size_t)buf * kTile, om.Rx + (size_t)(t + 2) * kTile, tile_bytes, &full[buf]);
        }
    }

#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int li = q * kThreads + threadIdx.x;
        const bool valid = li < nq;
        const float thr = b1[q] + win[q];
        // a third candidate chunk: the whole cloud, scanned by the warp together (one such
        // query at a time) rather than by its thread alone
        const bool whole = valid && b3[q] <= thr;
        float best = __int_as_float(0x7f800000);
        int bi = 0;
        if (valid && !whole) {
            int ca = c1[q], cb = c2[q];
            const bool two = b2[q] <= thr && cb != ca;
            if (two && cb < ca) { const int x = ca; ca = cb; cb = x; }
            exact_scan(om.R, ca * kChunk, min((ca + 1) * kChunk, om.M), sx[q], sy[q], sz[q], best, bi);
            if (two) exact_scan(om.R, cb * kChunk, min((cb + 1) * kChunk, om.M), sx[q], sy[q], sz[q], best, bi);
        }
        unsigned pending = __ballot_sync(0xffffffffu, whole);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1;
            float wb;
            int wi;
            warp_exact_all(om.R, om.M, __shfl_sync(0xffffffffu, sx[q], src), __shfl_sync(0xffffffffu, sy[q], src),
                           __shfl_sync(0xffffffffu, sz[q], src), wb, wi);
            if ((int)(threadIdx.x & 31) == src) { best = wb; bi = wi; }
        }
        if (!valid) continue;
        const long long g = q0 + li;
        a.nn_idx[g] = bi;
        if (a.dbg_d2) a.dbg_d2[g] = best;
        if (a.dbg_sp) {
            a.dbg_sp[g * 3 + 0] = sx[q];
            a.dbg_sp[g * 3 + 1] = sy[q];
            a.dbg_sp[g * 3 + 2] = sz[q];
        }
    }
    return true;
}

// match_pass with the smallest queries-per-thread count Q >= qn (Q <= QMAX).
template <class Shape, int QMAX>
__device__ __forceinline__ bool dispatch_pass(int qn, const FwdArgs &a, const ObjMeta &om, float4 fr, long long q0,
                                              int nq, ulonglong2 *tiles, unsigned long long *full,
                                              unsigned long long *never, int &seq, int *s_abort)
{
    if constexpr (QMAX > 1) {
        if (qn < QMAX) return dispatch_pass<Shape, QMAX - 1>(qn, a, om, fr, q0, nq, tiles, full, never, seq, s_abort);
    }
    return match_pass<Shape, QMAX>(a, om, fr, q0, nq, tiles, full, never, seq, s_abort);
}

// Persistent: CTA b runs the work items the host planned for it
// (cta_off[b] .. cta_off[b + 1] - 1, balanced by their cost), or without a plan
// items b, b + gridDim.x, ...; an item is at most kThreads * QPT queries of one
// object, and a partial item uses the smallest queries-per-thread
// instantiation that covers it.
template <class Shape>
__global__ void __launch_bounds__(Shape::kThreads, Shape::kMinBlocks) fwd_match_kernel(const FwdArgs a)
{
    constexpr int kThreads = Shape::kThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ulonglong2 *tiles = reinterpret_cast<ulonglong2 *>(smem_raw);
    __shared__ __align__(8) unsigned long long full[2], never;
    __shared__ int s_abort;
    const int it0 = a.cta_off ? a.cta_off[blockIdx.x] : blockIdx.x;
    const int it1 = a.cta_off ? a.cta_off[blockIdx.x + 1] : a.n_items;
    const int step = a.cta_off ? 1 : gridDim.x;
    if (it0 >= it1) return;
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long Qtot = (long long)a.L.T * a.L.N;
    int seq = 0;
    bool ok = true;
    for (int it = it0; it < it1 && ok; it += step) {
        FwdItem item;
        if (a.items) {
            item = a.items[it];
        } else {
            item.q0 = (long long)it * Shape::kItem;
            item.nq = (int)(Qtot - item.q0 < Shape::kItem ? Qtot - item.q0 : Shape::kItem);
            item.obj = 0;
        }
        const ObjMeta om = a.L.obj[item.obj];
        const float4 fr = a.L.frame[item.obj];
        const int qn = (item.nq + kThreads - 1) / kThreads;
        ok = dispatch_pass<Shape, Shape::QPT>(qn, a, om, fr, item.q0, item.nq, tiles, full, &never, seq, &s_abort);
    }
    if (!ok && threadIdx.x == 0)   // drain copies still in flight (bounded, full budget) before leaving
        for (int b = 0; b < 2; ++b) mbar_wait(&full[(seq + b) & 1], (unsigned)((seq + b) >> 1) & 1u);
}

using Shape0 = FwdShape<8, 64, 128, 2048, 3>;
using Shape1 = FwdShape<8, 32, 128, 2048, 3>;
using Shape2 = FwdShape<4, 64, 256, 2048, 2>;
using Shape3 = FwdShape<4, 32, 256, 2048, 2>;
using Shape4 = FwdShape<4, 64, 128, 1024, 5>;
using Shape5 = FwdShape<8, 64, 128, 1024, 4>;
using Shape6 = FwdShape<6, 64, 128, 1024, 4>;

template <class Shape>
int shape_grid()
{
    static int grid[kDeviceSlots] = {};
    static std::mutex mu;
    return per_device_value(grid, mu, [] {
        const int smem = 2 * Shape::kTile * 16;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(fwd_match_kernel<Shape>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_match_kernel<Shape>, Shape::kThreads, smem);
        return sms * (per_sm > 0 ? per_sm : 1);
    });
}

template <class Shape>
cudaError_t launch_shape(const FwdArgs &a, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)Shape::kTile * 16;
    fwd_match_kernel<Shape><<<shape_grid<Shape>(), Shape::kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// Apply f to the shape with index v (a default-constructed Shape tag).
template <class F>
auto with_shape(int v, F &&f)
{
    switch (v) {
        case 1: return f(Shape1{});
        case 2: return f(Shape2{});
        case 3: return f(Shape3{});
        case 4: return f(Shape4{});
        case 5: return f(Shape5{});
        case 6: return f(Shape6{});
        default: return f(Shape0{});
    }
}
constexpr int kTcVariant = 7;          // the tensor-core kernel (k_match_tc.cu)
static_assert(kFwdVariants == 8 && kTcVariant == kFwdVariants - 1, "shape table");
static_assert(Shape0::kItem == kFwdItemQueries, "unplanned launches use shape 0's items");

int fwd_shape_grid(int v)
{
    if (v == kTcVariant) return fwd_tc_grid();
    return with_shape(v, [](auto sh) { return shape_grid<decltype(sh)>(); });
}

int fwd_shape_threads(int v)
{
    if (v == kTcVariant) return fwd_tc_threads();
    return with_shape(v, [](auto sh) { return decltype(sh)::kThreads; });
}

int fwd_shape_queries(int v)
{
    if (v == kTcVariant) return fwd_tc_threads();     // one query per thread
    return with_shape(v, [](auto sh) { return decltype(sh)::kItem; });
}

int fwd_grid_size()
{
    int total = 0;
    for (int v = 0; v < kFwdVariants; ++v) total += fwd_shape_grid(v);
    return total;
}

const char *fwd_variant_name(int v)
{
    static const char *names[kFwdVariants] = {"qpt8-chunk64-t128-tile2048", "qpt8-chunk32-t128-tile2048",
                                              "qpt4-chunk64-t256-tile2048", "qpt4-chunk32-t256-tile2048",
                                              "qpt4-chunk64-t128-tile1024", "qpt8-chunk64-t128-tile1024",
                                              "qpt6-chunk64-t128-tile1024", "tc-f16x3-m128-n256"};
    return (v >= 0 && v < kFwdVariants) ? names[v] : "unknown";
}

cudaError_t launch_fwd_match(const FwdArgs &a, cudaStream_t st)
{
    if (a.variant == kTcVariant) return launch_fwd_match_tc(a, st);
    return with_shape(a.variant, [&](auto sh) { return launch_shape<decltype(sh)>(a, st); });
}

cudaError_t launch_fwd_exact(const FwdArgs &a, cudaStream_t st)
{
    return a.variant == kTcVariant ? launch_tc_exact(a, st) : cudaSuccess;
}

// Reference preparation for the screening stage (one CTA).  The frame: centre c =
// the midpoint of R's bounding box (float32), radius w = max |fl(r - c)| rounded
// up (float64 reduction); with compute_frame = false the given frame is kept (R
// is then a subset of the cloud the frame was made for, so its radius still
// bounds).  Layout: pairs of (-2 b, |b|^2) with b = fl(r - c), padded with
// (0, +inf) points to a whole number of tiles.
__global__ void ref_prep_kernel(const float4 *R, int M, int Mpad, ulonglong2 *Rx, float4 *frame, bool compute_frame)
{
    __shared__ double red[32];
    __shared__ float bmin[3][32], bmax[3][32];
    __shared__ float4 s_fr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    if (compute_frame) {
        float lo[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
        float hi[3] = {-lo[0], -lo[1], -lo[2]};
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
            const float4 r = R[i];
            lo[0] = fminf(lo[0], r.x); lo[1] = fminf(lo[1], r.y); lo[2] = fminf(lo[2], r.z);
            hi[0] = fmaxf(hi[0], r.x); hi[1] = fmaxf(hi[1], r.y); hi[2] = fmaxf(hi[2], r.z);
        }
        for (int k = 0; k < 3; ++k) {
            for (int o = 16; o > 0; o >>= 1) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
            if (lane == 0) { bmin[k][warp] = lo[k]; bmax[k][warp] = hi[k]; }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float c[3];
            for (int k = 0; k < 3; ++k) {
                float l = bmin[k][0], h = bmax[k][0];
                for (int w = 1; w < nw; ++w) { l = fminf(l, bmin[k][w]); h = fmaxf(h, bmax[k][w]); }
                c[k] = M > 0 ? 0.5f * l + 0.5f * h : 0.f;
            }
            s_fr = make_float4(c[0], c[1], c[2], 0.f);
        }
    } else if (threadIdx.x == 0) {
        s_fr = *frame;
    }
    __syncthreads();
    const float4 fr = s_fr;
    double m = 0.0;
    for (int q = threadIdx.x; q < Mpad / 2; q += blockDim.x) {
        float ax[2], ay[2], az[2], w[2];
        for (int k = 0; k < 2; ++k) {
            const int i = 2 * q + k;
            if (i < M) {
                const float4 r = R[i];
                const float bx = __fsub_rn(r.x, fr.x), by = __fsub_rn(r.y, fr.y), bz = __fsub_rn(r.z, fr.z);
                const double b2 = (double)bx * bx + (double)by * by + (double)bz * bz;
                m = fmax(m, b2);
                ax[k] = -2.f * bx; ay[k] = -2.f * by; az[k] = -2.f * bz;
                w[k] = (float)b2;
            } else {
                ax[k] = ay[k] = az[k] = 0.f;
                w[k] = __int_as_float(0x7f800000);
            }
        }
        // pair layout: point pair q -> {A, B} at 2 q, 2 q + 1 (any tile of an even
        // number of points is a contiguous range)
        ulonglong2 A, B;
        A.x = pack2(ax[0], ax[1]); A.y = pack2(ay[0], ay[1]);
        B.x = pack2(az[0], az[1]); B.y = pack2(w[0], w[1]);
        Rx[2 * (size_t)q] = A;
        Rx[2 * (size_t)q + 1] = B;
    }
    if (!compute_frame) return;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < nw; ++w) mm = fmax(mm, red[w]);
        *frame = make_float4(fr.x, fr.y, fr.z, (float)(sqrt(mm) * (1.0 + 1e-6)) + 1e-30f);
    }
}

cudaError_t launch_ref_prep(const float4 *R, int M, int Mpad, void *Rx, float4 *frame, bool compute_frame,
                            cudaStream_t st)
{
    ref_prep_kernel<<<1, 1024, 0, st>>>(R, M, Mpad, static_cast<ulonglong2 *>(Rx), frame, compute_frame);
    return cudaGetLastError();
}

}  // namespace asicp
