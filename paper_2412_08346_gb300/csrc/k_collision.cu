// Collision term: SDF test of the collision cloud in every particle's gripper
// frame (Eq. 12, Section IV-C) and the reverse matching of the colliding points
// onto the transformed contact cloud (Eq. 18).
#include "asicp_internal.cuh"

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
}  // namespace

// One CTA per particle: map every collision point c into the gripper frame,
// c' = R^T (c - t), interpolate the preshape's SDF and keep c when the value is
// > 0.  The colliding indices are compacted in ascending order (warp ballots
// and a block prefix), so results do not depend on scheduling.
__global__ void __launch_bounds__(kColThreads) collide_kernel(const CollideArgs a)
{
    __shared__ int swarp[kColThreads / 32];
    const int pk = blockIdx.x, p = pk / a.K;
    const float *th = a.theta + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2];
    float Rm[9];
    quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
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
            float val;
            hit = sdf_lookup(m, lx, ly, lz, val) && val > 0.f;
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

// One CTA per particle with colliding points: the particle's transformed contact
// cloud is built in shared memory with the same float32 transform as the
// forward matching, then each colliding point finds its nearest contact point
// (ties to the lowest index).  The float64 sums the collision cost and gradient
// are linear in are reduced per particle:
//   sum s (3), sum s s^T (xx,xy,xz,yy,yz,zz) (6), sum c (3), sum c s^T (9), sum |c|^2 (1)
// with s the matched gripper point in the gripper frame.
__global__ void __launch_bounds__(kColThreads) collide_nn_kernel(const CollideArgs a)
{
    extern __shared__ float4 sSp[];
    __shared__ double sred[kColThreads / 32][kColSums];
    const int pk = blockIdx.x, p = pk / a.K;
    const int n = a.ncol[pk];
    if (n == 0) return;
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
    for (int l = threadIdx.x; l < n; l += kColThreads) {
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
        acc[0] += sv[0]; acc[1] += sv[1]; acc[2] += sv[2];
        acc[3] = fma(sv[0], sv[0], acc[3]); acc[4] = fma(sv[0], sv[1], acc[4]); acc[5] = fma(sv[0], sv[2], acc[5]);
        acc[6] = fma(sv[1], sv[1], acc[6]); acc[7] = fma(sv[1], sv[2], acc[7]); acc[8] = fma(sv[2], sv[2], acc[8]);
        acc[9] += cv[0]; acc[10] += cv[1]; acc[11] += cv[2];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v) acc[12 + 3 * u + v] = fma(cv[u], sv[v], acc[12 + 3 * u + v]);
        acc[21] = fma(cv[0], cv[0], fma(cv[1], cv[1], fma(cv[2], cv[2], acc[21])));
    }
    warp_sum_f64(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < kColSums; ++c) sred[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < kColSums) {
        double s = 0.0;
        for (int w = 0; w < kColThreads / 32; ++w) s += sred[w][threadIdx.x];
        a.csums[(size_t)pk * kColSums + threadIdx.x] = s;
    }
}

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st)
{
    collide_kernel<<<a.PK, kColThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_collide_nn(const CollideArgs &a, cudaStream_t st)
{
    const size_t smem = sizeof(float4) * (size_t)a.N;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(collide_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    collide_nn_kernel<<<a.PK, kColThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace asicp
