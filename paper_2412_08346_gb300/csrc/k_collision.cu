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

// Block sum of double-float accumulators: warp trees in double-float, then the
// warps' partials added in float64 in warp order by NV threads.
template <int NV>
__device__ __forceinline__ void block_reduce_store(dfloat (&acc)[NV], double (*sred)[NV], double *out)
{
    warp_sum_df(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sred[warp][c] = (double)acc[c].hi + (double)acc[c].lo;
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
        dfloat acc[kFwdSums];
#pragma unroll
        for (int c = 0; c < kFwdSums; ++c) acc[c] = dfloat{0.f, 0.f};
        const float4 *S = a.S + (size_t)p * a.N;
        const int *idx = a.nn_idx + (size_t)pk * a.N;
        for (int i = threadIdx.x; i < a.N; i += kColThreads) {
            const float4 s = S[i];
            const float4 r = __ldg(a.R + idx[i]);
            const float rv[3] = {r.x, r.y, r.z}, sv[3] = {s.x, s.y, s.z};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                df_add(acc[u], rv[u]);
#pragma unroll
                for (int v = 0; v < 3; ++v) df_add_prod(acc[3 + 3 * u + v], rv[u], sv[v]);
                df_add_prod(acc[12], rv[u], rv[u]);
            }
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
    if (threadIdx.x == 0) {
        a.ncol[pk] = count;
        // queue this particle's chunks of colliding points for the reverse matching
        const int chunks = (a.Mc + kColChunk - 1) / kColChunk, used = (count + kColChunk - 1) / kColChunk;
        if (used > 0) {
            const int base = atomicAdd(&a.col_items[0], used);
            for (int c = 0; c < used; ++c) a.col_list[base + c] = pk * chunks + c;
        }
    }
}

// Persistent: CTAs take (particle, chunk of kColChunk colliding points) items
// from the list the collision kernel filled.  For an item the particle's
// transformed contact cloud is built in shared memory with the same float32
// transform as the forward matching; each warp then matches kQW colliding
// points against it (lanes stride over the contact points, a shuffle reduction
// picks the smallest distance, ties to the lowest index).  Per item, the sums
// the collision cost and gradient are linear in (double-float accumulation of
// exact products):
//   sum s (3), sum s s^T (xx,xy,xz,yy,yz,zz) (6), sum c (3), sum c s^T (9), sum |c|^2 (1)
// with s the matched gripper point in the gripper frame; the finalize kernel
// adds the chunks of a particle in chunk order, so the result does not depend
// on which CTA took which item.
__global__ void __launch_bounds__(kColThreads) collide_nn_kernel(const CollideArgs a)
{
    constexpr int kQW = kColChunk / (kColThreads / 32);     // colliding points per warp
    extern __shared__ float4 sSp[];
    __shared__ double sred[kColThreads / 32][kColSums];
    __shared__ int s_item;
    const int chunks = (a.Mc + kColChunk - 1) / kColChunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.col_items[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.col_items[0]) break;
        const int code = a.col_list[item];
        const int pk = code / chunks, chunk = code - pk * chunks, p = pk / a.K;
        const int n = a.ncol[pk];
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
        const int l0 = chunk * kColChunk + warp * kQW;
        float cx[kQW], cy[kQW], cz[kQW], best[kQW];
        int bi[kQW];
#pragma unroll
        for (int q = 0; q < kQW; ++q) {
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l0 + q < n) c = a.C[a.colidx[(size_t)pk * a.Mc + l0 + q]];
            cx[q] = c.x; cy[q] = c.y; cz[q] = c.z;
            best[q] = __int_as_float(0x7f800000);
            bi[q] = 0;
        }
        for (int i = lane; i < a.N; i += 32) {
            const float4 s = sSp[i];
#pragma unroll
            for (int q = 0; q < kQW; ++q) {
                const float d = dist2_f32(s.x, s.y, s.z, cx[q], cy[q], cz[q]);
                if (d < best[q]) { best[q] = d; bi[q] = i; }
            }
        }
#pragma unroll
        for (int q = 0; q < kQW; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best[q], o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi[q], o);
                if (ob < best[q] || (ob == best[q] && oi < bi[q])) { best[q] = ob; bi[q] = oi; }
            }
        dfloat acc[kColSums];
#pragma unroll
        for (int c = 0; c < kColSums; ++c) acc[c] = dfloat{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kQW; ++q) {
            if (lane != q || l0 + q >= n) continue;       // lane q records colliding point q
            if (a.dbg_colnn) a.dbg_colnn[(size_t)pk * a.Mc + l0 + q] = bi[q];
            const float4 s = S[bi[q]];
            const float sv[3] = {s.x, s.y, s.z}, cv[3] = {cx[q], cy[q], cz[q]};
            acc[0] = dfloat{sv[0], 0.f}; acc[1] = dfloat{sv[1], 0.f}; acc[2] = dfloat{sv[2], 0.f};
            df_add_prod(acc[3], sv[0], sv[0]); df_add_prod(acc[4], sv[0], sv[1]); df_add_prod(acc[5], sv[0], sv[2]);
            df_add_prod(acc[6], sv[1], sv[1]); df_add_prod(acc[7], sv[1], sv[2]); df_add_prod(acc[8], sv[2], sv[2]);
            acc[9] = dfloat{cv[0], 0.f}; acc[10] = dfloat{cv[1], 0.f}; acc[11] = dfloat{cv[2], 0.f};
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) df_add_prod(acc[12 + 3 * u + v], cv[u], sv[v]);
            df_add_prod(acc[21], cv[0], cv[0]); df_add_prod(acc[21], cv[1], cv[1]); df_add_prod(acc[21], cv[2], cv[2]);
        }
        block_reduce_store<kColSums>(acc, sred, a.csums + ((size_t)pk * chunks + chunk) * kColSums);
        __syncthreads();   // sSp, sred and s_item are reused by the next item
    }
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
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = 4 * sms;
    }
    const size_t smem = sizeof(float4) * (size_t)a.N;
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
