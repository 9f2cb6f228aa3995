// Per-particle matching sums and the collision term: SDF test of the
// collision cloud in every particle's gripper frame (Eq. 12, Section IV-C) and
// the reverse matching of the colliding points onto the transformed contact
// cloud (Eq. 18).
#include "asicp_internal.cuh"

#include <climits>

namespace asicp {

namespace {
constexpr int kColThreads = 256;       // reverse matching
constexpr int kTestThreads = 128;      // collision test: one CTA per particle, small enough that every
                                       // particle of a paper-scale launch is resident at once
constexpr int kColU = 4;          // collision points per thread per compaction round
constexpr int kPairB = 4;         // matching pairs per thread whose loads overlap (57.5 us per paper-scale
                                  // launch against 61.8 us one pair at a time; 72 registers, 7 CTAs per SM)

// Trilinear interpolation of a node-centred grid at gripper-frame point (x, y, z).
// Returns false when the point lies outside the grid's node box (the grid covers
// the gripper, so such a point is not inside it).  The eight corner values come
// from the corner-packed copy of the grid: one 32-byte record per cell, read as
// two float4 from a single 32-byte sector.
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
    const float4 *cell = m.cells + 2 * ((size_t)ix + (size_t)(m.nx - 1) * ((size_t)iy + (size_t)(m.ny - 1) * iz));
    const float4 z0 = __ldg(cell), z1 = __ldg(cell + 1);
    const float c000 = z0.x, c100 = z0.y, c010 = z0.z, c110 = z0.w;
    const float c001 = z1.x, c101 = z1.y, c011 = z1.z, c111 = z1.w;
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
        for (int w = 0; w < kTestThreads / 32; ++w) s += sred[w][threadIdx.x];
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
__global__ void __launch_bounds__(kTestThreads) collide_kernel(const CollideArgs a)
{
    if (a.err && *a.err != kDevOk) return;    // the matching gave up: its correspondences are not valid
    __shared__ int swarp[kColU][kTestThreads / 32];
    __shared__ double sred[kTestThreads / 32][kFwdSums];
    const int pk = blockIdx.x;
    const int grp = a.L.part_grp[pk], p = grp % a.L.P;
    const ObjMeta om = a.L.obj[grp / a.L.P];
    const int N = a.L.N, Mc = om.Mc;
    const float *th = a.theta + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2];
    float Rm[9];
    quat_rot_f32(th[3], th[4], th[5], th[6], Rm);

    {
        dfloat acc[kFwdSums];
#pragma unroll
        for (int c = 0; c < kFwdSums; ++c) acc[c] = dfloat{0.f, 0.f};
        const float4 *S = a.S + (size_t)p * N;
        const int *idx = a.nn_idx + (size_t)pk * N;
        auto add_pair = [&](float4 r, float4 s) {
            const float rv[3] = {r.x, r.y, r.z}, sv[3] = {s.x, s.y, s.z};
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                df_add(acc[u], rv[u]);
#pragma unroll
                for (int v = 0; v < 3; ++v) df_add_prod(acc[3 + 3 * u + v], rv[u], sv[v]);
                df_add_prod(acc[12], rv[u], rv[u]);
            }
        };
        // kPairB pairs per thread at a time: their index loads, then their object-point loads,
        // are in flight together (the pairs are still added in the same order)
        int i = threadIdx.x;
        for (; i + (kPairB - 1) * kTestThreads < N; i += kPairB * kTestThreads) {
            int id[kPairB];
            float4 s[kPairB], r[kPairB];
#pragma unroll
            for (int u = 0; u < kPairB; ++u) { id[u] = idx[i + u * kTestThreads]; s[u] = S[i + u * kTestThreads]; }
#pragma unroll
            for (int u = 0; u < kPairB; ++u) r[u] = __ldg(om.R + id[u]);
#pragma unroll
            for (int u = 0; u < kPairB; ++u) add_pair(r[u], s[u]);
        }
        for (; i < N; i += kTestThreads) add_pair(__ldg(om.R + idx[i]), S[i]);
        block_reduce_store<kFwdSums>(acc, sred, a.fsums + (size_t)pk * kFwdSums);
    }

    const SdfMeta m = a.meta[p];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *colidx = a.colidx + om.colidx_base + (long long)(pk - om.pfirst) * Mc;
    int count = 0;
    // kU points per thread per round (their loads and lookups overlap), one
    // compaction per round in ascending point order (round slot, warp, lane)
    for (int c0 = 0; c0 < Mc; c0 += kTestThreads * kColU) {
        float4 v[kColU];
#pragma unroll
        for (int u = 0; u < kColU; ++u) {
            const int c = c0 + u * kTestThreads + threadIdx.x;
            v[u] = c < Mc ? om.C[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bool hit[kColU];
#pragma unroll
        for (int u = 0; u < kColU; ++u) {
            const int c = c0 + u * kTestThreads + threadIdx.x;
            hit[u] = false;
            if (c < Mc) {
                const float dx = __fsub_rn(v[u].x, tx), dy = __fsub_rn(v[u].y, ty), dz = __fsub_rn(v[u].z, tz);
                const float lx = __fmaf_rn(Rm[0], dx, __fmaf_rn(Rm[3], dy, __fmul_rn(Rm[6], dz)));
                const float ly = __fmaf_rn(Rm[1], dx, __fmaf_rn(Rm[4], dy, __fmul_rn(Rm[7], dz)));
                const float lz = __fmaf_rn(Rm[2], dx, __fmaf_rn(Rm[5], dy, __fmul_rn(Rm[8], dz)));
                if (lx >= m.lo[0] && lx <= m.hi[0] && ly >= m.lo[1] && ly <= m.hi[1] && lz >= m.lo[2] &&
                    lz <= m.hi[2]) {
                    float val;
                    hit[u] = sdf_lookup(m, lx, ly, lz, val) && val > 0.f;
                }
            }
        }
        unsigned bal[kColU];
#pragma unroll
        for (int u = 0; u < kColU; ++u) {
            bal[u] = __ballot_sync(0xffffffffu, hit[u]);
            if (lane == 0) swarp[u][warp] = __popc(bal[u]);
        }
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int u = 0; u < kColU; ++u) {
            int mine = 0;
#pragma unroll
            for (int w = 0; w < kTestThreads / 32; ++w) {
                const int n = swarp[u][w];
                mine += w < warp ? n : 0;
                tot += n;
            }
            if (hit[u])
                colidx[count + before + mine + __popc(bal[u] & ((1u << lane) - 1u))] = c0 + u * kTestThreads + threadIdx.x;
            before = tot;
        }
        count += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.ncol[pk] = count;
        // queue this particle's chunks of colliding points for the reverse matching
        const int used = (count + kColChunk - 1) / kColChunk;
        if (used > 0) {
            const int base = atomicAdd(&a.col_items[0], used);
            for (int c = 0; c < used; ++c) {
                a.col_list[2 * (base + c)] = pk;
                a.col_list[2 * (base + c) + 1] = c;
            }
        }
    }
}

namespace {
__device__ __forceinline__ unsigned long long pk2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Total order of float32 values (no NaN) as unsigned keys, and back.
__device__ __forceinline__ unsigned ord_key(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_val(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// (best, bi) <- the smaller of itself and the partner lane's, ties to the lower index.
__device__ __forceinline__ void argmin_xor(float &best, int &bi, int o)
{
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
}

// Operands of the collision sums: sum index -> (a, b) as indices into a
// colliding point's record {s_x, s_y, s_z, c_x, c_y, c_z, 1, 0}; sum 21 (|c|^2)
// adds the three squares of c.
__constant__ unsigned char kColSel[kColSums][2] = {
    {0, 6}, {1, 6}, {2, 6},                                  // sum s
    {0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2},          // sum s s^T (upper triangle)
    {3, 6}, {4, 6}, {5, 6},                                  // sum c
    {3, 0}, {3, 1}, {3, 2}, {4, 0}, {4, 1}, {4, 2}, {5, 0}, {5, 1}, {5, 2},   // sum c s^T
    {3, 3}};                                                 // sum |c|^2
}  // namespace

// Persistent: CTAs take (particle, chunk of kColChunk colliding points) items
// from the list the collision kernel filled.  Per item the particle's
// transformed contact cloud S' is built in shared memory twice, both arranged
// by lane chunks (chunk l = points l + 32 k): in the screening layout
// (-2 s', |s'|^2), point pairs (l + 64 m, l + 32 + 64 m) at slot 32 m + l, and
// exact (float4), chunk l contiguous with a stride of KC + 1 (no bank
// conflicts).  Each warp matches kQW colliding points c:
//  1. screening, relative to the particle's translation t (so the error does not
//     grow with the distance from the origin): with b = fl(s' - t) and
//     a = fl(c - t), lane l evaluates d~ = |b|^2 - 2 a.b over chunk l (packed
//     f32x2 FMAs, 3-input min); warp min-reductions give the best chunk minimum
//     b1 (lane l1, the lowest on ties) and the best of the other chunks b2;
//  2. exact choice: with delta = u (9 B^2 + 10.1 A B) bounding the error of d~
//     against |c - s'|^2 + const (B = max |b|, A = |a|: the float32 evaluation
//     within u (7 B^2 + 6.1 A B), the rounding of a and b within u (2 B^2 + 4 A B)
//     beyond a term that does not depend on s'), the nearest point lies in chunk
//     l1 unless b2 <= b1 + 2 delta; four lanes per colliding point re-evaluate chunk l1 with the
//     exact-form distance, ties to the lowest index; in the rare other case the
//     warp scans the whole cloud that way.
// The sums the collision cost and gradient are linear in are then accumulated
// per item (double-float, exact products) by 8 threads per sum over 8
// colliding points each, merged in a fixed tree:
//   sum s (3), sum s s^T (xx,xy,xz,yy,yz,zz) (6), sum c (3), sum c s^T (9), sum |c|^2 (1)
// with s the matched gripper point in the gripper frame; the finalize kernel adds
// the chunks of a particle in chunk order, so the result does not depend on
// which CTA took which item.
__global__ void __launch_bounds__(kColThreads) collide_nn_kernel(const CollideArgs a)
{
    if (a.err && *a.err != kDevOk) return;
    constexpr int kWarps = kColThreads / 32;
    constexpr int kQW = kColChunk / kWarps;                  // colliding points per warp
    static_assert(kQW == 8 && kColChunk == 64, "lane groups of four per colliding point");
    static_assert(kColSums * 8 <= kColThreads, "eight threads per sum");
    extern __shared__ __align__(16) unsigned char smem_nn[];
    const int N = a.L.N;
    const int Npad = (N + 63) / 64 * 64;
    const int KC = Npad / 32, KCs = KC + 1;                  // points per lane chunk, exact-layout stride
    ulonglong2 *sXA = reinterpret_cast<ulonglong2 *>(smem_nn);             // [Npad/2] {-2x pair}{-2y pair}
    ulonglong2 *sXB = sXA + Npad / 2;                                      // [Npad/2] {-2z pair}{w pair}
    float4 *sE = reinterpret_cast<float4 *>(sXB + Npad / 2);               // [32][KC + 1] exact S'
    __shared__ float4 sC[kColChunk];                          // colliding points of the item
    __shared__ float sRec[kColChunk][8];                      // {s, c, 1, 0} per matched colliding point
    __shared__ int s_item;
    __shared__ float s_smax[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slots = Npad / 64;                 // point pairs per lane
    // Two barriers per item.  Thread 0 takes the next item right after the first
    // (its index is read at the top of the loop, after the second).  After the
    // second barrier the transformed cloud and sC are no longer read, so the
    // next item may overwrite them while slower threads still add this item's
    // sums; those read only sRec, which the next item writes after its own
    // first barrier.
    if (threadIdx.x == 0) s_item = atomicAdd(&a.col_items[1], 1);
    __syncthreads();
    for (;;) {
        const int item = s_item;
        if (item >= a.col_items[0]) break;
        const int pk = a.col_list[2 * item], chunk = a.col_list[2 * item + 1];
        const int grp = a.L.part_grp[pk], p = grp % a.L.P;
        const ObjMeta om = a.L.obj[grp / a.L.P];
        const int n = a.ncol[pk];
        const int *colidx = a.colidx + om.colidx_base + (long long)(pk - om.pfirst) * om.Mc;
        const int l0 = chunk * kColChunk;
        const float *th = a.theta + (size_t)pk * 8;
        const float tx = th[0], ty = th[1], tz = th[2];
        float Rm[9];
        quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
        const float4 *S = a.S + (size_t)p * N;
        if (threadIdx.x < kColChunk) {
            const int j = threadIdx.x;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l0 + j < n) c = om.C[colidx[l0 + j]];
            sC[j] = c;
        }
        float smax2 = 0.f;
        for (int q = threadIdx.x; q < Npad / 2; q += kColThreads) {
            const int l = q & 31, m = q >> 5;
            float ax[2], ay[2], az[2], w[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = l + 32 * h + 64 * m;
                float4 e = make_float4(__int_as_float(0x7f800000), __int_as_float(0x7f800000),
                                       __int_as_float(0x7f800000), 0.f);
                if (r < N) {
                    const float4 sv = S[r];
                    const float3 o = xform_f32(Rm, tx, ty, tz, sv.x, sv.y, sv.z);
                    e = make_float4(o.x, o.y, o.z, 0.f);
                    const float bx = __fsub_rn(o.x, tx), by = __fsub_rn(o.y, ty), bz = __fsub_rn(o.z, tz);
                    ax[h] = -2.f * bx; ay[h] = -2.f * by; az[h] = -2.f * bz;
                    w[h] = __fmaf_rn(bx, bx, __fmaf_rn(by, by, __fmul_rn(bz, bz)));
                    smax2 = fmaxf(smax2, w[h]);
                } else {
                    ax[h] = ay[h] = az[h] = 0.f;
                    w[h] = __int_as_float(0x7f800000);
                }
                sE[l * KCs + 2 * m + h] = e;
            }
            ulonglong2 A, B;
            A.x = pk2(ax[0], ax[1]); A.y = pk2(ay[0], ay[1]);
            B.x = pk2(az[0], az[1]); B.y = pk2(w[0], w[1]);
            sXA[q] = A;
            sXB[q] = B;
        }
        for (int o = 16; o > 0; o >>= 1) smax2 = fmaxf(smax2, __shfl_xor_sync(0xffffffffu, smax2, o));
        if (lane == 0) s_smax[warp] = smax2;
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&a.col_items[1], 1);
        float sm2 = 0.f;
        for (int w8 = 0; w8 < kWarps; ++w8) sm2 = fmaxf(sm2, s_smax[w8]);
        const float smax = sqrtf(sm2) * 1.0001f;

        // colliding points of this warp (warp-uniform): a warp whose eight slots are all past the
        // particle's count (the padding of its last item) skips the matching; its records are zeros
        const int g = lane >> 2, gs = lane & 3;       // lane group g works on colliding point g
        const float4 cq = sC[warp * kQW + g];
        float best = __int_as_float(0x7f800000);
        int bi = 0x7fffffff;
        if (l0 + warp * kQW < n) {
            // 1. screening of this warp's colliding points, lane l over chunk l
            unsigned long long qx[kQW], qy[kQW], qz[kQW];
            float cm[kQW];
#pragma unroll
            for (int q = 0; q < kQW; ++q) {
                const float4 c = sC[warp * kQW + q];
                const float ax = __fsub_rn(c.x, tx), ay = __fsub_rn(c.y, ty), az = __fsub_rn(c.z, tz);
                qx[q] = pk2(ax, ax); qy[q] = pk2(ay, ay); qz[q] = pk2(az, az);
                cm[q] = __int_as_float(0x7f800000);
            }
            for (int m = 0; m < slots; ++m) {
                const ulonglong2 A = sXA[m * 32 + lane];
                const ulonglong2 B = sXB[m * 32 + lane];
#pragma unroll
                for (int q = 0; q < kQW; ++q) {
                    const unsigned long long d = ffma2(qx[q], A.x, ffma2(qy[q], A.y, ffma2(qz[q], B.x, B.y)));
                    float d0, d1;
                    upk2(d, d0, d1);
                    cm[q] = fmin3(cm[q], d0, d1);
                }
            }
            // best chunk l1 (lowest lane on ties) and whether another chunk may hold the nearest point
            int my_l1 = 0;
            unsigned full_scan = 0u;
#pragma unroll
            for (int q = 0; q < kQW; ++q) {
                const unsigned key = ord_key(cm[q]);
                const unsigned k1 = __reduce_min_sync(0xffffffffu, key);
                const int l1 = __ffs(__ballot_sync(0xffffffffu, key == k1)) - 1;
                const unsigned k2 = __reduce_min_sync(0xffffffffu, lane == l1 ? 0xffffffffu : key);
                const float4 c = sC[warp * kQW + q];
                const float ax = __fsub_rn(c.x, tx), ay = __fsub_rn(c.y, ty), az = __fsub_rn(c.z, tz);
                const float cn = sqrtf(ax * ax + ay * ay + az * az) * 1.001f;
                const float win = 2.02f * 5.9604645e-8f * (9.f * smax * smax + 10.1f * cn * smax);
                if (key_val(k2) <= key_val(k1) + win) full_scan |= 1u << q;
                if (g == q) my_l1 = l1;
            }
            // 2. exact choice: four lanes per colliding point over its chunk l1
            for (int k = gs; k < KC; k += 4) {
                const int r = my_l1 + 32 * k;
                if (r >= N) break;
                const float4 e = sE[my_l1 * KCs + k];
                const float d = dist2_f32(e.x, e.y, e.z, cq.x, cq.y, cq.z);
                if (d < best) { best = d; bi = r; }
            }
            argmin_xor(best, bi, 1);
            argmin_xor(best, bi, 2);
            if (bi >= N) bi = 0;     // no finite distance at all (not reached with finite inputs)
            // rare: the whole cloud, lane l over chunk l
            while (full_scan) {
                const int q = __ffs(full_scan) - 1;
                full_scan &= full_scan - 1;
                const float4 c = sC[warp * kQW + q];
                float fb = __int_as_float(0x7f800000);
                int fi = 0x7fffffff;
                for (int k = 0; k < KC; ++k) {
                    const int r = lane + 32 * k;
                    if (r >= N) break;
                    const float4 e = sE[lane * KCs + k];
                    const float d = dist2_f32(e.x, e.y, e.z, c.x, c.y, c.z);
                    if (d < fb) { fb = d; fi = r; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) argmin_xor(fb, fi, o);
                if (g == q) { best = fb; bi = fi < N ? fi : 0; }
            }
        }
        if (gs == 0) {
            const int j = warp * kQW + g;
            const bool valid = l0 + j < n;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                s = S[bi];
                if (a.dbg_colnn) a.dbg_colnn[om.colidx_base + (long long)(pk - om.pfirst) * om.Mc + l0 + j] = bi;
            }
            sRec[j][0] = s.x; sRec[j][1] = s.y; sRec[j][2] = s.z;
            sRec[j][3] = valid ? cq.x : 0.f; sRec[j][4] = valid ? cq.y : 0.f; sRec[j][5] = valid ? cq.z : 0.f;
            sRec[j][6] = valid ? 1.f : 0.f; sRec[j][7] = 0.f;
        }
        __syncthreads();
        // 3. the item's sums: thread (sum e, part) adds colliding points part + 8 u, u = 0 .. 7
        if (threadIdx.x < (kColSums * 8 + 31) / 32 * 32) {
            const int e = threadIdx.x >> 3, part = threadIdx.x & 7;
            dfloat acc{0.f, 0.f};
            if (e < kColSums) {
                const int ia = kColSel[e][0], ib = kColSel[e][1];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float *rec = sRec[part + 8 * u];
                    df_add_prod(acc, rec[ia], rec[ib]);
                    if (e == kColSums - 1) {
                        df_add_prod(acc, rec[4], rec[4]);
                        df_add_prod(acc, rec[5], rec[5]);
                    }
                }
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                dfloat y;
                y.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
                y.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
                df_merge(acc, y);
            }
            if (part == 0 && e < kColSums)
                a.csums[(om.csum_base + (long long)(pk - om.pfirst) * om.chunks + chunk) * kColSums + e] =
                    (double)acc.hi + (double)acc.lo;
        }
    }
}

cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st)
{
    collide_kernel<<<a.L.T, kTestThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t init_collision_attributes()
{
    return cudaFuncSetAttribute(collide_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(float4) * kMaxN + 32 * sizeof(float4)));
}

cudaError_t launch_collide_nn(const CollideArgs &a, cudaStream_t st)
{
    static int grids[kDeviceSlots] = {};
    static std::mutex mu;
    const int grid = per_device_value(grids, mu, [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return 4 * sms;
    });
    const size_t smem = 2 * sizeof(float4) * (size_t)((a.L.N + 63) / 64 * 64) + 32 * sizeof(float4);
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

// Corner-packed copy of a grid: cell (ix, iy, iz), x fastest over the
// (nx-1)(ny-1)(nz-1) cells, gets its eight corner values as two float4.
__global__ void sdf_pack_cells_kernel(const float *grid, int nx, int ny, int nz, float4 *cells)
{
    const long long nc = (long long)(nx - 1) * (ny - 1) * (nz - 1);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(c % (nx - 1)), iy = (int)((c / (nx - 1)) % (ny - 1)), iz = (int)(c / ((long long)(nx - 1) * (ny - 1)));
        const float *g = grid + (size_t)ix + (size_t)nx * ((size_t)iy + (size_t)ny * iz);
        const size_t sy = nx, sz = (size_t)nx * ny;
        cells[2 * c] = make_float4(g[0], g[1], g[sy], g[sy + 1]);
        cells[2 * c + 1] = make_float4(g[sz], g[sz + 1], g[sz + sy], g[sz + sy + 1]);
    }
}

size_t sdf_cells_bytes(int nx, int ny, int nz) { return 2 * sizeof(float4) * (size_t)(nx - 1) * (ny - 1) * (nz - 1); }

cudaError_t launch_sdf_pack_cells(const float *grid, int nx, int ny, int nz, float4 *cells, cudaStream_t st)
{
    const long long nc = (long long)(nx - 1) * (ny - 1) * (nz - 1);
    long long blocks = (nc + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    sdf_pack_cells_kernel<<<(int)blocks, 256, 0, st>>>(grid, nx, ny, nz, cells);
    return cudaGetLastError();
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
