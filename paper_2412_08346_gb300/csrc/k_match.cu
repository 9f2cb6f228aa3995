// Forward matching: transform + brute-force nearest neighbour + per-particle sums.
//
// For particle (p, j) and gripper point i the kernel forms s'_i = R_j s_i + t_j
// (Algorithm 1, "transform the source cloud") and finds the object point with
// the smallest squared distance, ties to the lowest index (Eq. 1).  The object
// cloud is streamed through shared memory in tiles; every thread keeps QPT
// queries in registers, so one broadcast shared-memory read of a reference point
// feeds QPT distance evaluations.
//
// Instead of per-point residuals the epilogue accumulates, in float64, the
// sums that the cost and gradient of Eqs. 13-17 are linear in:
//   sum r_i (3), sum r_i s_i^T (9), sum |r_i|^2 (1)
// where r_i is the matched object point and s_i the untransformed gripper point.
// Both are float32, so every product is exact in float64; the update kernel
// rebuilds sum e_i, sum e_i s_i^T and sum |e_i|^2 (e_i = R s_i + t - r_i) from
// them in float64 without the rounding of float32 residuals.
#include "asicp_internal.cuh"

namespace asicp {

namespace {
constexpr int QPT = 4;   // queries per thread
}

int fwd_queries_per_block() { return kFwdThreads * QPT; }

__global__ void __launch_bounds__(kFwdThreads) fwd_match_kernel(const FwdArgs a)
{
    __shared__ float4 sR[kRefTile];
    __shared__ double sred[kFwdThreads / 32][kFwdSums];

    const int pk = blockIdx.y;
    const int p = pk / a.K;
    const int blk = blockIdx.x;
    const float *th = a.theta + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2];
    float Rm[9];
    quat_rot_f32(th[3], th[4], th[5], th[6], Rm);

    const int base = blk * kFwdThreads * QPT + threadIdx.x;
    float qx[QPT], qy[QPT], qz[QPT], best[QPT];
    int bi[QPT];
#pragma unroll
    for (int q = 0; q < QPT; ++q) {
        const int i = base + q * kFwdThreads;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < a.N) s = a.S[(size_t)p * a.N + i];
        const float3 o = xform_f32(Rm, tx, ty, tz, s.x, s.y, s.z);
        qx[q] = o.x; qy[q] = o.y; qz[q] = o.z;
        best[q] = __int_as_float(0x7f800000);   // +inf
        bi[q] = 0;
    }

    for (int r0 = 0; r0 < a.M; r0 += kRefTile) {
        const int n = min(kRefTile, a.M - r0);
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += kFwdThreads) sR[r] = a.R[r0 + r];
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < n; ++r) {
            const float4 ref = sR[r];
#pragma unroll
            for (int q = 0; q < QPT; ++q) {
                const float d = dist2_f32(qx[q], qy[q], qz[q], ref.x, ref.y, ref.z);
                if (d < best[q]) { best[q] = d; bi[q] = r0 + r; }
            }
        }
    }

    double acc[kFwdSums];
#pragma unroll
    for (int c = 0; c < kFwdSums; ++c) acc[c] = 0.0;
#pragma unroll
    for (int q = 0; q < QPT; ++q) {
        const int i = base + q * kFwdThreads;
        if (i < a.N) {
            const float4 s = a.S[(size_t)p * a.N + i];
            const float4 r = a.R[bi[q]];
            const double rv[3] = {r.x, r.y, r.z}, sv[3] = {s.x, s.y, s.z};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                acc[u] += rv[u];
#pragma unroll
                for (int v = 0; v < 3; ++v) acc[3 + 3 * u + v] = fma(rv[u], sv[v], acc[3 + 3 * u + v]);
            }
            acc[12] = fma(rv[0], rv[0], fma(rv[1], rv[1], fma(rv[2], rv[2], acc[12])));
            const size_t o = (size_t)pk * a.N + i;
            if (a.dbg_idx) a.dbg_idx[o] = bi[q];
            if (a.dbg_d2) a.dbg_d2[o] = best[q];
            if (a.dbg_sp) {
                a.dbg_sp[o * 3 + 0] = qx[q];
                a.dbg_sp[o * 3 + 1] = qy[q];
                a.dbg_sp[o * 3 + 2] = qz[q];
            }
        }
    }
    warp_sum_f64(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < kFwdSums; ++c) sred[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < kFwdSums) {
        double s = 0.0;
        for (int w = 0; w < kFwdThreads / 32; ++w) s += sred[w][threadIdx.x];
        a.fsums[((size_t)pk * a.nb + blk) * kFwdSums + threadIdx.x] = s;
    }
}

cudaError_t launch_fwd_match(const FwdArgs &a, cudaStream_t st)
{
    dim3 grid(a.nb, a.PK);
    fwd_match_kernel<<<grid, kFwdThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace asicp
