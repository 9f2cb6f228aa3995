// Per-particle matching sums and the collision term: SDF test of the
// collision cloud in every particle's gripper frame (Eq. 12, Section IV-C) and
// the reverse matching of the colliding points onto the transformed contact
// cloud (Eq. 18).
#include "asicp_internal.cuh"

#include <climits>

namespace asicp {

namespace {
constexpr int kColThreads = 256;

// Trilinear interpolation of a node-centred grid at gripper-frame point (x, y, z).
// Returns false when the point lies outside the grid's node box (the grid covers
// the gripper, so such a point is not inside it).
__device__ __forceinline__ bool sdf_lookup(const SdfMeta &m, float x, float y, float z, float &val)
{
    const float ux = __fdiv_rn(__fsub_rn(x, m.ox), m.voxel);
    const float uy = __fdiv_rn(__fsub_rn(y, m.oy), m.voxel);
    const float uz = __fdiv_rn(__fsub_rn(z, m.oz), m.voxel);
    if (!(ux >= 0.f && ux <= (float)(m.nx - 1) && uy >= 0.f && uy <= (float)(m.ny - 1) &&
          uz >= 0.f && uz <= (float)(m.nz - 1)))
        return false;
    const int ix = min((int)floorf(ux), m.nx - 2);
    const int iy = min((int)floorf(uy), m.ny - 2);
    const int iz = min((int)floorf(uz), m.nz - 2);
    const float fx = ux - (float)ix, fy = uy - (float)iy, fz = uz - (float)iz;
    const float *g = m.grid + (size_t)ix + (size_t)m.nx * ((size_t)iy + (size_t)m.ny * iz);
    const size_t sy = m.nx, sz = (size_t)m.nx * m.ny;
    const float c000 = __ldg(g), c100 = __ldg(g + 1);
    const float c010 = __ldg(g + sy), c110 = __ldg(g + sy + 1);
    const float c001 = __ldg(g + sz), c101 = __ldg(g + sz + 1);
    const float c011 = __ldg(g + sz + sy), c111 = __ldg(g + sz + sy + 1);
    const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
    val = gx * gy * gz * c000 + fx * gy * gz * c100 + gx * fy * gz * c010 + fx * fy * gz * c110 +
          gx * gy * fz * c001 + fx * gy * fz * c101 + gx * fy * fz * c011 + fx * fy * fz * c111;
    return true;
}

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], double (*sred)[NV], double *out)
{
    warp_sum_f64(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sred[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < kColThreads / 32; ++w) s += sred[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}
}  // namespace

// One CTA per particle.
//  1. Matching sums of the forward pairs (i <-> nn_idx[i]) in float64:
//     sum r (3), sum r s^T (9), sum |r|^2 (1), r the matched object point and s the
//     gripper point in the gripper frame (exact products of float32 values).
//  2. Collision test: every collision point c is mapped into the gripper frame,
//     c' = R^T (c - t); points outside the box of cells with a positive corner
//     cannot interpolate to a positive value and are skipped; the others are
//     looked up in the preshape's SDF and kept when the value is > 0.  The
//     colliding indices are compacted in ascending order (warp ballots and a
//     block prefix), so results do not depend on scheduling.
__global__ void __launch_bounds__(kColThreads) collide_kernel(const CollideArgs a)
{
    __shared__ int swarp[kColThreads / 32];
    __shared__ double sred[kColThreads / 32][kFwdSums];
    const int pk = blockIdx.x, p = pk / a.K;
    const float *th = a.theta + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2];
    float Rm[9];
    quat_rot_f32(th[3], th[4], th[5], th[6], Rm);

    {
        double acc[kFwdSums];
#pragma unroll
        for (int c = 0; c < kFwdSums; ++c) acc[c] = 0.0;
        const float4 *S = a.S + (size_t)p * a.N;
        const int *idx = a.nn_idx + (size_t)pk * a.N;
        for (int i = threadIdx.x; i < a.N; i += kColThreads) {
            const float4 s = S[i];
            const float4 r = __ldg(a.R + idx[i]);
            const double rv[3] = {r.x, r.y, r.z}, sv[3] = {s.x, s.y, s.z};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                acc[u] += rv[u];
#pragma unroll
                for (int v = 0; v < 3; ++v) acc[3 + 3 * u + v] = fma(rv[u], sv[v], acc[3 + 3 * u + v]);
            }
            acc[12] = fma(rv[0], rv[0], fma(rv[1], rv[1], fma(rv[2], rv[2], acc[12])));
        }
        block_reduce_store<kFwdSums>(acc, sred, a.fsums + (size_t)pk * kFwdSums);
    }

    const SdfMeta m = a.meta[p];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int count = 0;
    for (int c0 = 0; c0 < a.Mc; c0 += kColThreads) {
        const int c = c0 + threadIdx.x;
        bool hit = false;
        if (c < a.Mc) {
            const float4 v = a.C[c];
            const float dx = __fsub_rn(v.x, tx), dy = __fsub_rn(v.y, ty), dz = __fsub_rn(v.z, tz);
            const float lx = __fmaf_rn(Rm[0], dx, __fmaf_rn(Rm[3], dy, __fmul_rn(Rm[6], dz)));
            const float ly = __fmaf_rn(Rm[1], dx, __fmaf_rn(Rm[4], dy, __fmul_rn(Rm[7], dz)));
            const float lz = __fmaf_rn(Rm[2], dx, __fmaf_rn(Rm[5], dy, __fmul_rn(Rm[8], dz)));
            if (lx >= m.lo[0] && lx <= m.hi[0] && ly >= m.lo[1] && ly <= m.hi[1] && lz >= m.lo[2] && lz <= m.hi[2]) {
                float val;
                hit = sdf_lookup(m, lx, ly, lz, val) && val > 0.f;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) swarp[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kColThreads / 32; ++w) {
            const int n = swarp[w];
            off += w < warp ? n : 0;
            tot += n;
        }
        if (hit) a.colidx[(size_t)pk * a.Mc + count + off + __popc(bal & ((1u << lane) - 1u))] = c;
        count += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ncol[pk] = count;
}

// Grid (particle, chunk of kColChunk colliding points); chunks past the
// particle's colliding count exit at once.  The particle's transformed contact
// cloud is built in shared memory with the same float32 transform as the
// forward matching, then each colliding point finds its nearest contact point
// (ties to the lowest index).  Per chunk, the float64 sums the collision cost
// and gradient are linear in:
//   sum s (3), sum s s^T (xx,xy,xz,yy,yz,zz) (6), sum c (3), sum c s^T (9), sum |c|^2 (1)
// with s the matched gripper point in the gripper frame; the update kernel adds
// the chunks in order.
__global__ void __launch_bounds__(kColThreads) collide_nn_kernel(const CollideArgs a)
{
    extern __shared__ float4 sSp[];
    __shared__ double sred[kColThreads / 32][kColSums];
    const int pk = blockIdx.x, p = pk / a.K;
    const int n = a.ncol[pk];
    const int l0 = blockIdx.y * kColChunk;
    if (l0 >= n) return;
    const float *th = a.theta + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2];
    float Rm[9];
    quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
    const float4 *S = a.S + (size_t)p * a.N;
    for (int i = threadIdx.x; i < a.N; i += kColThreads) {
        const float4 s = S[i];
        const float3 o = xform_f32(Rm, tx, ty, tz, s.x, s.y, s.z);
        sSp[i] = make_float4(o.x, o.y, o.z, 0.f);
    }
    __syncthreads();
    double acc[kColSums];
#pragma unroll
    for (int c = 0; c < kColSums; ++c) acc[c] = 0.0;
    const int l = l0 + threadIdx.x;
    if (l < n) {
        const float4 c = a.C[a.colidx[(size_t)pk * a.Mc + l]];
        float best = __int_as_float(0x7f800000);
        int bi = 0;
        for (int i = 0; i < a.N; ++i) {
            const float4 s = sSp[i];
            const float d = dist2_f32(s.x, s.y, s.z, c.x, c.y, c.z);
            if (d < best) { best = d; bi = i; }
        }
        if (a.dbg_colnn) a.dbg_colnn[(size_t)pk * a.Mc + l] = bi;
        const float4 s = S[bi];
        const double sv[3] = {s.x, s.y, s.z}, cv[3] = {c.x, c.y, c.z};
        acc[0] = sv[0]; acc[1] = sv[1]; acc[2] = sv[2];
        acc[3] = sv[0] * sv[0]; acc[4] = sv[0] * sv[1]; acc[5] = sv[0] * sv[2];
        acc[6] = sv[1] * sv[1]; acc[7] = sv[1] * sv[2]; acc[8] = sv[2] * sv[2];
        acc[9] = cv[0]; acc[10] = cv[1]; acc[11] = cv[2];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v) acc[12 + 3 * u + v] = cv[u] * sv[v];
        acc[21] = fma(cv[0], cv[0], fma(cv[1], cv[1], cv[2] * cv[2]));
    }
    const int nchunks = (a.Mc + kColChunk - 1) / kColChunk;
    block_reduce_store<kColSums>(acc, sred, a.csums + ((size_t)pk * nchunks + blockIdx.y) * kColSums);
}

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st)
{
    collide_kernel<<<a.PK, kColThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t init_collision_attributes()
{
    return cudaFuncSetAttribute(collide_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float4) * kMaxN));
}

cudaError_t launch_collide_nn(const CollideArgs &a, cudaStream_t st)
{
    const size_t smem = sizeof(float4) * (size_t)a.N;
    dim3 grid(a.PK, (a.Mc + kColChunk - 1) / kColChunk);
    collide_nn_kernel<<<grid, kColThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// Index box of the grid nodes with a positive value: box6 = (min x, min y, min z,
// max x, max y, max z); the caller initialises it to (INT_MAX x3, INT_MIN x3).
__global__ void sdf_box_kernel(const float *grid, int nx, int ny, int nz, int *box6)
{
    const long long n = (long long)nx * ny * nz;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (grid[i] > 0.f) {
            const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
            lo[0] = min(lo[0], x); lo[1] = min(lo[1], y); lo[2] = min(lo[2], z);
            hi[0] = max(hi[0], x); hi[1] = max(hi[1], y); hi[2] = max(hi[2], z);
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (lo[a] != INT_MAX) atomicMin(box6 + a, lo[a]);
        if (hi[a] != INT_MIN) atomicMax(box6 + 3 + a, hi[a]);
    }
}

cudaError_t launch_sdf_box(const float *grid, int nx, int ny, int nz, int *box6, cudaStream_t st)
{
    const long long n = (long long)nx * ny * nz;
    long long blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    sdf_box_kernel<<<(int)blocks, 256, 0, st>>>(grid, nx, ny, nz, box6);
    return cudaGetLastError();
}

}  // namespace asicp
