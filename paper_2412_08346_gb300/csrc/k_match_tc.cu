// Forward matching on the tensor cores: tcgen05 f16 MMAs with split operands.
//
// The screening value of the float32 kernel, d~(r) = |b|^2 - 2 a.b with a and b
// the query and the object point relative to the object's frame centre c (Eq. 1
// up to the query's own |a|^2 and a term that does not depend on r), is a
// contraction of an augmented query row with an augmented object-point column.
// Coordinates are scaled by a power of two lam (lam B in (128, 256], B = max |b|),
// every scaled factor is split into two f16 parts (x = x_h + x_l, rounded to
// nearest) and lam^2 |b|^2 / 4 into three, so that with alpha = -2 lam a and
// rho = lam b
//     A row    = [alpha_h, alpha_h, alpha_l, 4, 4, 4, 2^15, 0, 0, 0]      (K = 16)
//     B column = [rho_h, rho_l, rho_h, w_1, w_2, w_3, 0, 0, 0, 0]
// gives A.B = lam^2 (|b|^2 - 2 a.b) up to rounding: one kind::f16 MMA per 128
// queries x COLS object points, accumulated in float32 in tensor memory.
// (Slot 12 is 2^15 for padding columns, which then never screen in.)
//
// Error bound, u = 2^-24, in lam^2 units, A = |a|: the dropped alpha_l.rho_l and
// the rounding of the low parts are at most 3 * 2^-22 |alpha_k| |rho_k| per
// coordinate (f16 has an 11-bit significand), i.e. 24 u A |b| in all;
// w = fl(lam^2 |b|^2) is within u lam^2 |b|^2; products of f16 values are exact
// in float32, and the tensor core's float32 accumulation is taken to stay within
// 16 u of the sum of the magnitudes of its addends (<= 1.002 (|b|^2 + 2 A |b|));
// measured on GB300: at most 2.9 u over 10^6 random rows of this form.  Low parts
// below the f16 normal range (2^-14) add at most 2^-14 * 1.74 lam (2 A + |b|)
// even if flushed, and the last part of w / 4 at most 2^-12.  The rounding of
// a = fl(s' - c) and b = fl(r - c) adds, beyond a term that does not depend on r,
// at most u (2 B^2 + 4 A B) (as in the float32 kernel).  So
//     delta_tc = u lam^2 (20 B^2 + 61 A B) + 2^-14 * 1.74 lam (2 A + B) + 2^-12
// bounds the error of the screening value against lam^2 |s' - r|^2 + const.  A
// query whose scaled coordinates would leave the f16 range takes the whole-cloud
// scan.  Each query keeps its kTop best chunk minima (chunks of 64 object points)
// and the best of the rest; the chunks within 2 delta_tc of the best are
// rescanned with the exact-form float32 distance (ties to the lower index) by
// tc_exact_kernel, eight lanes per query, or, when more than kTop qualify, by a
// warp scanning the whole cloud for that query together.  The result is the
// exact-form argmin over every point that can be nearest, as in the float32
// kernel.
//
// Per CTA: work items of 128 queries (one per tensor-memory lane = query row of
// the MMA); object tiles of COLS points (already in the MMA's shared-memory
// layout) stream through a ring of kStages buffers by 1D bulk copies.  One thread
// issues the copies and another the MMAs: every mbarrier, copy or MMA operation of
// a single thread costs on the order of a hundred cycles (measured with clock64
// stamps on GB300), so one thread doing both set the pace, and a wide tile with a
// single MMA and a single commit amortises those operations over more pairs.  A
// tcgen05.ld.red per 64 columns returns a chunk minimum directly.  Each CTA has one
// COLS-column accumulator; the 512 / COLS CTAs of an SM (COLS tensor-memory
// columns each) take turns on the tensor pipe and overlap one another's per-item
// prologue.  The per-tile chain of handoffs (copy landed, MMA issue and commit,
// completion seen by the reduction warps, tensor-memory loads, accumulator
// released) sets the pace, not the tensor pipe; every mbarrier wait (150-200 cycles
// even on a completed phase), arrival, MMA issue or commit adds to it.  Measured
// slower: splitting a tile's MMA into parts with their own commits, reading the
// accumulator with more warps, narrower tiles with two or four accumulators per CTA
// (each tile pays the fixed cost of a wait, a first load and a handoff), and the
// reduction warps issuing the MMAs after a CTA barrier (the issue from a warp, and
// the barrier, cost more than the dedicated thread's wake-up).  Every wait is bounded: on expiry the kernel reports ASICP_ERR_TIMEOUT
// through the error word, drains its own copies and MMAs (bounded), frees its
// tensor memory and returns.
#include "asicp_internal.cuh"
#include "async_copy.cuh"
#include "tcgen05.cuh"

#include <cstdint>
#include <cuda_fp16.h>

namespace asicp {

namespace {

constexpr int kRows = 128;                 // queries per item = MMA M = tensor-memory lanes
constexpr int kCols = 256;                 // object points per tile of the prepared layout
constexpr int kQueries = kRows;            // queries per item = reduction threads (one warp per quadrant)
constexpr int kThreadsTc = kQueries + 64;  // + one warp for the copies, one for the MMAs
constexpr int kAug = 16;                   // augmented length (one K = 16 MMA)
constexpr int kStages = 10;                // object tiles in flight
constexpr int kChunk = 64;                 // screening chunk = columns per tcgen05.ld.red
constexpr int kTop = 4;                    // chunks per query the exact stage rescans at most
constexpr unsigned kTileBytes = kCols * kAug * 2;       // 8 KB
constexpr unsigned kABytes = kRows * kAug * 2;          // 4 KB of query rows
constexpr unsigned kLBO = 128, kSBO = 256; // core matrices (8 rows x 16 B): K-adjacent 128 B, row groups 256 B
static_assert(kRefTilePts % kCols == 0, "object padding must be whole tiles");
static_assert(kCols % kChunk == 0, "whole chunks per tile");
// The first COLS < kCols rows of a prepared tile are themselves a tile of COLS points in
// the same layout (8-row groups are contiguous), so kernels with narrower tiles read
// the same buffer.
template <int COLS>
constexpr size_t tc_smem_bytes() { return (size_t)kABytes + (size_t)kStages * (COLS * kAug * 2); }

// byte offset of element (row, k) in the no-swizzle K-major layout
__host__ __device__ constexpr unsigned core_offset(int row, int k) { return kmajor_offset(row, k, kLBO, kSBO); }

__device__ __forceinline__ uint64_t smem_desc(unsigned addr) { return tc_smem_desc(addr, kLBO, kSBO); }

// Power-of-two scale lam with lam B in (128, 256] (B clamped below at 2^-30),
// so that scaled coordinates and |b|^2 / 4 fit the f16 range.
__device__ __forceinline__ float tc_scale(float B)
{
    int ex;
    frexpf(fmaxf(B, 9.3132257e-10f), &ex);
    return ldexpf(1.f, 8 - ex);
}

// Minimum over the 64 accumulator columns at taddr of this thread's lane: the
// tcgen05.ld.red and its wait in one statement, so the compiler sees the
// destination registers written when the statement ends.
__device__ __forceinline__ float ld_min64(uint32_t taddr)
{
    uint32_t v[64];
    float m;
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x64.min.f32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, %64, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63]), "=f"(m)
        : "r"(taddr)
        : "memory");
    return m;
}

// Write the query row of global query g (valid or not) of an item on the object with
// frame fr into the row buffer sA at row `row`; returns the screening window 2 delta_tc
// in lam^2 units (+inf for a query the f16 split cannot represent, so that it takes
// the whole-cloud scan).
__device__ __forceinline__ float build_query_row(const FwdArgs &a, long long g, bool valid, float4 fr,
                                                 unsigned char *sA, int row)
{
    float3 o = make_float3(0.f, 0.f, 0.f);
    if (valid) {
        const int pk = (int)(g / a.L.N), i = (int)(g - (long long)pk * a.L.N);
        const int pre = a.L.part_grp[pk] % a.L.P;
        const float *th = a.theta + (size_t)pk * 8;
        float Rm[9];
        quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
        const float4 s = a.S[(size_t)pre * a.L.N + i];
        o = xform_f32(Rm, th[0], th[1], th[2], s.x, s.y, s.z);
    }
    // the query relative to the frame centre (a = fl(s' - c))
    o = make_float3(__fsub_rn(o.x, fr.x), __fsub_rn(o.y, fr.y), __fsub_rn(o.z, fr.z));
    // alpha = -2 lam a in two f16 parts, unless a part would leave the f16 range
    const float lam = tc_scale(fr.w);
    const float c[3] = {-2.f * lam * o.x, -2.f * lam * o.y, -2.f * lam * o.z};
    const bool far = !(fabsf(c[0]) < 65000.f && fabsf(c[1]) < 65000.f && fabsf(c[2]) < 65000.f);
    __half v[kAug];
    for (int k = 0; k < kAug; ++k) v[k] = __float2half_rn(0.f);
    if (!far) {
        for (int k = 0; k < 3; ++k) {
            const __half h = __float2half_rn(c[k]);
            v[k] = h; v[3 + k] = h; v[6 + k] = __float2half_rn(c[k] - __half2float(h));
        }
    }
    v[9] = v[10] = v[11] = __float2half_rn(4.f);
    v[12] = __float2half_rn(32768.f);
    for (int j = 0; j < kAug / 8; ++j) {
        uint4 pk;
        pk.x = (uint32_t)__half_as_ushort(v[8 * j + 0]) | ((uint32_t)__half_as_ushort(v[8 * j + 1]) << 16);
        pk.y = (uint32_t)__half_as_ushort(v[8 * j + 2]) | ((uint32_t)__half_as_ushort(v[8 * j + 3]) << 16);
        pk.z = (uint32_t)__half_as_ushort(v[8 * j + 4]) | ((uint32_t)__half_as_ushort(v[8 * j + 5]) << 16);
        pk.w = (uint32_t)__half_as_ushort(v[8 * j + 6]) | ((uint32_t)__half_as_ushort(v[8 * j + 7]) << 16);
        *reinterpret_cast<uint4 *>(sA + core_offset(row, 8 * j)) = pk;
    }
    const float an = sqrtf(o.x * o.x + o.y * o.y + o.z * o.z) * 1.001f;
    // 2 delta_tc in lam^2 units (1 % margin for evaluating the bound in float32)
    return far ? __int_as_float(0x7f800000)
               : 2.02f * (5.9604645e-8f * lam * lam * (20.f * fr.w * fr.w + 61.f * an * fr.w) +
                          6.1035156e-5f * 1.74f * lam * (2.f * an + fr.w) + 2.45e-4f);
}

}  // namespace

// Augmented object tiles for the tensor-core kernel: point r goes to tile
// r / kCols, row r % kCols of that tile's MMA layout, as f16 parts of lam b and
// lam^2 |b|^2 / 4 with b = fl(r - c) (frame centre c, lam from the frame radius);
// padding points (r >= M) carry only 2^15 in slot 12, which meets 2^15 in every
// query row: + 2^30, so they never screen in.
__global__ void tc_ref_prep_kernel(const float4 *R, int M, int Mpad, const float4 *frame, __half *Rt)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Mpad) return;
    const float4 fr = *frame;
    const float lam = tc_scale(fr.w);
    __half v[kAug];
    for (int k = 0; k < kAug; ++k) v[k] = __float2half_rn(0.f);
    if (r < M) {
        const float4 p = R[r];
        const float c[3] = {lam * __fsub_rn(p.x, fr.x), lam * __fsub_rn(p.y, fr.y), lam * __fsub_rn(p.z, fr.z)};
        for (int k = 0; k < 3; ++k) {
            const __half h = __float2half_rn(c[k]);
            const __half l = __float2half_rn(c[k] - __half2float(h));
            v[k] = h; v[3 + k] = l; v[6 + k] = h;
        }
        // w = fl(lam^2 |b|^2) / 4, split into three f16 parts (exact to 2^-33 relative)
        const double w = (double)(float)((double)c[0] * c[0] + (double)c[1] * c[1] + (double)c[2] * c[2]) * 0.25;
        const __half w1 = __float2half_rn((float)w);
        const __half w2 = __float2half_rn((float)(w - (double)__half2float(w1)));
        const __half w3 = __float2half_rn((float)(w - (double)__half2float(w1) - (double)__half2float(w2)));
        v[9] = w1; v[10] = w2; v[11] = w3;
    } else {
        v[12] = __float2half_rn(32768.f);
    }
    unsigned char *tile = reinterpret_cast<unsigned char *>(Rt) + (size_t)(r / kCols) * kTileBytes;
    for (int k = 0; k < kAug; ++k) *reinterpret_cast<__half *>(tile + core_offset(r % kCols, k)) = v[k];
}

cudaError_t launch_tc_ref_prep(const float4 *R, int M, int Mpad, const float4 *frame, void *Rt, cudaStream_t st)
{
    tc_ref_prep_kernel<<<(Mpad + 255) / 256, 256, 0, st>>>(R, M, Mpad, frame, static_cast<__half *>(Rt));
    return cudaGetLastError();
}

size_t tc_ref_bytes(int Mpad) { return (size_t)Mpad / kCols * kTileBytes; }

// Warp roles: warps 0-3 (one query per thread; warp w reads TMEM lanes
// 32 w .. 32 w + 31) build the augmented query rows, read the accumulator and keep
// the candidate chunks; lane 0 of warp 4 streams the object tiles, lane 0 of warp 5
// issues the MMAs (one per tile of COLS points).  They meet on mbarriers only (no
// CTA-wide barrier inside the loop):
//   bfull[s]  tile in stage s has landed          (copy -> MMA)
//   bempty[s] the MMA reading stage s is done:     (MMA commit -> copy, and -> reduction:
//             the accumulator holds that tile     its next phase needs the reduction's acce)
//   acce      the accumulator has been read        (reduction -> MMA, one arrival per warp)
//   afull     the item's query rows are written    (reduction warps -> MMA, one arrival per warp)
// COLS: tile width = accumulator columns; 512 / COLS CTAs per SM share the 512
// tensor-memory columns (256: two; 128-column tiles with four CTAs per SM
// measured slower, their registers capped at 80).
template <int COLS>
__global__ void __launch_bounds__(kThreadsTc, 512 / COLS) fwd_match_tc_kernel(const FwdArgs a)
{
    static_assert(COLS == 128 || COLS == 256, "tile width");
    constexpr uint32_t kIdesc = tc_idesc_f16(false, COLS, kRows);
    constexpr unsigned kTile = COLS * kAug * 2;
    constexpr int kTileChunks = COLS / kChunk;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char *sA = smem_tc;                               // [kABytes] query rows
    unsigned char *sB = smem_tc + kABytes;                     // [kStages][kTile] object tiles
    __shared__ __align__(8) unsigned long long bfull[kStages], bempty[kStages], acce, afull;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int it0 = a.cta_off ? a.cta_off[blockIdx.x] : blockIdx.x;
    const int it1 = a.cta_off ? a.cta_off[blockIdx.x + 1] : a.n_items;
    const int step = a.cta_off ? 1 : gridDim.x;
    if (it0 >= it1) return;
    const long long Qtot = (long long)a.L.T * a.L.N;
    auto item_at = [&](int it) {
        FwdItem item;
        if (a.items) {
            item = a.items[it];
        } else {
            item.q0 = (long long)it * kQueries;
            item.nq = (int)(Qtot - item.q0 < kQueries ? Qtot - item.q0 : kQueries);
            item.obj = 0;
        }
        return item;
    };
    auto fail = [&]() {
        if (!s_abort) atomicExch(a.err, kDevTimeout);
        s_abort = 1;
    };

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s) { mbar_init(&bfull[s], 1); mbar_init(&bempty[s], 1); }
        // one arrival per reduction warp (its lane 0, after the warp's loads or stores)
        mbar_init(&acce, kQueries / 32);
        mbar_init(&afull, kQueries / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc_alloc(&s_tmem, COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == kQueries / 32) {
        // ------------------------------------------------ object-tile copies (one thread)
        if (lane == 0) {
            // copies issued so far, the stage of the next one and the parity of the ring's lap
            int p_seq = 0, p_stage = 0;
            unsigned p_lap = 0u;
            bool ok = true;
            for (int it = it0; it < it1 && ok; it += step) {
                const ObjMeta &om = a.L.obj[item_at(it).obj];
                const unsigned char *src = reinterpret_cast<const unsigned char *>(om.Rt);
                const int ntiles = om.Mpad / COLS;
                for (int t = 0; t < ntiles; ++t) {
                    // the stage is free once the MMA of its previous tile is done
                    if (s_abort || !mbar_wait(&bempty[p_stage], p_lap ^ 1u)) { ok = false; break; }
                    mbar_arrive_tx(&bfull[p_stage], kTile);
                    bulk_load(sB + (size_t)p_stage * kTile, src + (size_t)t * kTile, kTile, &bfull[p_stage]);
                    ++p_seq;
                    if (++p_stage == kStages) { p_stage = 0; p_lap ^= 1u; }
                }
            }
            if (!ok) {
                fail();
                // drain (bounded): the last copy issued into each stage
                for (int q = p_seq > kStages ? p_seq - kStages : 0; q < p_seq; ++q)
                    mbar_wait(&bfull[q % kStages], (unsigned)((q / kStages) & 1));
            }
        }
    } else if (warp == kQueries / 32 + 1) {
        // ------------------------------------------------ MMAs (one thread)
        if (lane == 0) {
            // tiles consumed so far, their stage and the parity of the ring's lap (kept
            // incrementally: no division on this thread's path)
            int seq = 0, c_stage = 0, last_stage = -1;
            unsigned c_lap = 0u, last_lap = 0u;
            int ia = 0;
            for (int it = it0; it < it1 && !s_abort; it += step, ++ia) {
                const int ntiles = a.L.obj[item_at(it).obj].Mpad / COLS;
                // the item's query rows are written
                if (!mbar_wait(&afull, (unsigned)(ia & 1))) { fail(); break; }
                tc_fence_after();
                for (int t = 0; t < ntiles; ++t, ++seq) {
                    const int stage = c_stage;
                    if (s_abort || !mbar_wait(&bfull[stage], c_lap) || !mbar_wait(&acce, ((unsigned)seq & 1u) ^ 1u)) {
                        fail();
                        break;
                    }
                    tc_fence_after();
                    const unsigned a0 = smem_u32(sA), b0 = smem_u32(sB + (size_t)stage * kTile);
                    tc_mma_f16(tmem, smem_desc(a0), smem_desc(b0), kIdesc, 0u);
                    // one commit per tile: its completion frees the stage for the copy thread and
                    // hands the accumulator to the reduction warps
                    tc_commit(&bempty[stage]);
                    last_stage = stage;
                    last_lap = c_lap;
                    if (++c_stage == kStages) { c_stage = 0; c_lap ^= 1u; }
                }
            }
            // drain (bounded): the MMAs issued (the last commit tracks the earlier ones)
            if (s_abort && last_stage >= 0) mbar_wait(&bempty[last_stage], last_lap);
        }
    } else {
        // ------------------------------------------------ query rows, reduction, exact choice
        const int row = tid;                               // query row = TMEM lane
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        int r_stage = 0;          // stage and lap of the next tile, as on the MMA thread
        unsigned r_lap = 0u;
        for (int it = it0; it < it1; it += step) {
            if (__any_sync(0xffffffffu, s_abort)) break;
            // the item's query rows (the previous item's MMAs are complete: its last
            // accumulator was waited for); only the screening window lives through the tiles
            const int ntiles = a.L.obj[item_at(it).obj].Mpad / COLS;
            const FwdItem item = item_at(it);
            const float win = build_query_row(a, item.q0 + tid, tid < item.nq, a.L.frame[item.obj], sA, row);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull);
            // the kTop best chunk minima (ascending) with their chunk ids, and the best of the rest
            float bk[kTop], brest = __int_as_float(0x7f800000);
            int ck[kTop];
#pragma unroll
            for (int k = 0; k < kTop; ++k) { bk[k] = __int_as_float(0x7f800000); ck[k] = 0; }
            bool good = true;
            for (int t = 0; t < ntiles; ++t) {
                // the tile's MMA is complete once its stage barrier has flipped
                good = mbar_wait_warp(&bempty[r_stage], r_lap);
                if (++r_stage == kStages) { r_stage = 0; r_lap ^= 1u; }
                if (!__all_sync(0xffffffffu, good && !s_abort)) { good = false; break; }
                tc_fence_after();
                float mv[kTileChunks];
#pragma unroll
                for (int h = 0; h < kTileChunks; ++h) {
                    const uint32_t ta = tmem + lane_base + (uint32_t)(h * kChunk);
                    mv[h] = ld_min64(ta);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce);
#pragma unroll
                for (int h = 0; h < kTileChunks; ++h) {
                    // insert (v, chunk gc); strict < keeps the earlier chunk first on equal minima
                    float v = mv[h];
                    int gc = t * kTileChunks + h;
#pragma unroll
                    for (int k = 0; k < kTop; ++k) {
                        const bool lt = v < bk[k];
                        const float bv = bk[k];
                        const int cv = ck[k];
                        bk[k] = lt ? v : bv;
                        ck[k] = lt ? gc : cv;
                        v = lt ? bv : v;
                        gc = lt ? cv : gc;
                    }
                    brest = fminf(brest, v);
                }
            }
            if (!good) { fail(); break; }

            // the chunks that can hold the nearest point (within 2 delta_tc of the best), or
            // the whole cloud when more than kTop qualify; tc_exact_kernel rescans them
            const float thr = bk[0] + win;
            if (tid < item.nq) {
                int4 cd;
                if (brest <= thr) {
                    cd = make_int4(-2, -1, -1, -1);
                } else {
                    cd.x = ck[0];
                    cd.y = bk[1] <= thr ? ck[1] : -1;
                    cd.z = bk[2] <= thr ? ck[2] : -1;
                    cd.w = bk[3] <= thr ? ck[3] : -1;
                }
                a.cand[item.q0 + tid] = cd;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, COLS);
    }
}

// Exact choice after the tensor-core screening.  Each warp takes 32 consecutive
// queries; eight lanes rescan one query's candidate chunks together (lane l of the
// group reads points l, l + 8, ..., so every load instruction reads four whole
// 128-byte lines), four queries at a time, and three xor-shuffle rounds inside the
// group give the smallest exact-form float32 distance with the lowest index
// holding it.  Distances are non-negative (or +inf), so their bits order as
// unsigned integers; NaN (only from non-finite poses) orders above +inf and is
// never chosen.  A query marked for the whole cloud is scanned by the warp
// together.  Separate from the screening kernel so that these loads do not stall
// the tensor pipe between work items.  The transformed point is recomputed with
// the same float32 operations as in the screening kernel, so it is the same value.

// Merge this lane's (key, index) into the warp's running best (wk, wi), ties to
// the lower index; every lane ends with the same (wk, wi).
__device__ __forceinline__ void warp_merge_min(unsigned key, int idx, unsigned &wk, int &wi)
{
    const unsigned m = __reduce_min_sync(0xffffffffu, key);
    const int mi = (int)__reduce_min_sync(0xffffffffu, key == m ? (unsigned)idx : 0x7fffffffu);
    if (m < wk || (m == wk && mi < wi)) { wk = m; wi = mi; }
}

// (key, index) of the nearest point of chunk c for this lane's share (points
// c * kChunk + sub + 8 k), merged into (bk, bi) with ties to the lower index.
__device__ __forceinline__ void group_chunk(const float4 *__restrict__ R, int M, int c, int sub, float qx, float qy,
                                            float qz, unsigned &bk, int &bi)
{
    const int base = c * kChunk + sub;
    unsigned ck = 0x7f800000u;
    int ci = 0x7fffffff;
    if ((c + 1) * kChunk <= M) {
#pragma unroll
        for (int k = 0; k < kChunk / 8; ++k) {
            const float4 v = __ldg(R + base + 8 * k);
            const unsigned kk = __float_as_uint(dist2_f32(qx, qy, qz, v.x, v.y, v.z));
            if (kk < ck) { ck = kk; ci = base + 8 * k; }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kChunk / 8; ++k) {
            const int r = base + 8 * k;
            const float4 v = __ldg(R + min(r, M - 1));
            const unsigned kk = r < M ? __float_as_uint(dist2_f32(qx, qy, qz, v.x, v.y, v.z)) : 0x7f800000u;
            if (kk < ck) { ck = kk; ci = r; }
        }
    }
    if (ck < bk || (ck == bk && ci < bi)) { bk = ck; bi = ci; }
}

__global__ void __launch_bounds__(256) tc_exact_kernel(const FwdArgs a)
{
    if (*a.err != kDevOk) return;     // the screening gave up: its candidates are not valid
    const long long Qtot = (long long)a.L.T * a.L.N;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long wq0 = g - (threadIdx.x & 31);     // first query of this warp
    const bool valid = g < Qtot;
    const int lane = threadIdx.x & 31, grp = lane >> 3, sub = lane & 7;
    float3 o = make_float3(0.f, 0.f, 0.f);
    int obj = 0;
    int4 cd = make_int4(-1, -1, -1, -1);
    if (valid) {
        const int pk = (int)(g / a.L.N), i = (int)(g - (long long)pk * a.L.N);
        const int grp_id = a.L.part_grp[pk];
        obj = grp_id / a.L.P;
        const float *th = a.theta + (size_t)pk * 8;
        float Rm[9];
        quat_rot_f32(th[3], th[4], th[5], th[6], Rm);
        const float4 s = a.S[(size_t)(grp_id % a.L.P) * a.L.N + i];
        o = xform_f32(Rm, th[0], th[1], th[2], s.x, s.y, s.z);
        cd = a.cand[g];
        if (a.dbg_sp) {
            a.dbg_sp[g * 3 + 0] = o.x;
            a.dbg_sp[g * 3 + 1] = o.y;
            a.dbg_sp[g * 3 + 2] = o.z;
        }
    }
    // candidate chunks: four queries at a time, eight lanes each
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
        const int src = it * 8 + grp * 2;                  // two queries per group and round
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int q = src + half;
            const float qx = __shfl_sync(0xffffffffu, o.x, q), qy = __shfl_sync(0xffffffffu, o.y, q),
                        qz = __shfl_sync(0xffffffffu, o.z, q);
            const int qo = __shfl_sync(0xffffffffu, obj, q);
            const int c0 = __shfl_sync(0xffffffffu, cd.x, q), c1 = __shfl_sync(0xffffffffu, cd.y, q),
                      c2 = __shfl_sync(0xffffffffu, cd.z, q), c3 = __shfl_sync(0xffffffffu, cd.w, q);
            const bool qv = wq0 + q < Qtot && c0 >= 0;      // valid and not a whole-cloud query
            unsigned bk = 0x7f800000u;
            int bi = 0x7fffffff;
            int M = 1;
            if (qv) {
                const float4 *R = a.L.obj[qo].R;
                M = a.L.obj[qo].M;
                group_chunk(R, M, c0, sub, qx, qy, qz, bk, bi);
                if (c1 >= 0) group_chunk(R, M, c1, sub, qx, qy, qz, bk, bi);
                if (c2 >= 0) group_chunk(R, M, c2, sub, qx, qy, qz, bk, bi);
                if (c3 >= 0) group_chunk(R, M, c3, sub, qx, qy, qz, bk, bi);
            }
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const unsigned ok = __shfl_xor_sync(0xffffffffu, bk, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ok < bk || (ok == bk && oi < bi)) { bk = ok; bi = oi; }
            }
            if (qv && sub == 0) {
                a.nn_idx[wq0 + q] = bk < 0x7f800000u && bi < M ? bi : 0;   // no finite distance: 0
                if (a.dbg_d2) a.dbg_d2[wq0 + q] = __uint_as_float(bk < 0x7f800000u ? bk : 0x7f800000u);
            }
        }
    }
    // whole-cloud queries, one at a time by the warp together
    unsigned pending = __ballot_sync(0xffffffffu, valid && cd.x == -2);
    while (pending) {
        const int src = __ffs(pending) - 1;
        pending &= pending - 1;
        const float qx = __shfl_sync(0xffffffffu, o.x, src), qy = __shfl_sync(0xffffffffu, o.y, src),
                    qz = __shfl_sync(0xffffffffu, o.z, src);
        const int qo = __shfl_sync(0xffffffffu, obj, src);
        const float4 *R = a.L.obj[qo].R;
        const int M = a.L.obj[qo].M;
        unsigned k = 0x7f800000u;
        int ki = 0x7fffffff;
        for (int r = lane; r < M; r += 32) {
            const float4 v = __ldg(R + r);
            const unsigned dk = __float_as_uint(dist2_f32(qx, qy, qz, v.x, v.y, v.z));
            if (dk < k) { k = dk; ki = r; }
        }
        unsigned wk = 0x7f800000u;
        int wi = 0x7fffffff;
        warp_merge_min(k, ki, wk, wi);
        if (lane == src) {
            a.nn_idx[g] = wk < 0x7f800000u && wi < M ? wi : 0;
            if (a.dbg_d2) a.dbg_d2[g] = __uint_as_float(wk);
        }
    }
}

constexpr int kTcCols = 256;               // the kernel's tile width (accumulator columns)

// 512 / COLS CTAs per SM: each allocates COLS of the 512 tensor-memory columns,
// and the shared-memory request leaves no room for more.
int fwd_tc_grid()
{
    static int grid[kDeviceSlots] = {};
    static std::mutex mu;
    return per_device_value(grid, mu, [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(fwd_match_tc_kernel<kTcCols>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes<kTcCols>());
        cudaFuncSetAttribute(fwd_match_tc_kernel<kTcCols>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        return (512 / kTcCols) * sms;
    });
}

int fwd_tc_threads() { return kQueries; }

cudaError_t launch_fwd_match_tc(const FwdArgs &a, cudaStream_t st)
{
    fwd_match_tc_kernel<kTcCols><<<fwd_tc_grid(), kThreadsTc, tc_smem_bytes<kTcCols>(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_exact(const FwdArgs &a, cudaStream_t st)
{
    const long long Qtot = (long long)a.L.T * a.L.N;
    if (Qtot == 0) return cudaSuccess;
    tc_exact_kernel<<<(unsigned)((Qtot + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace asicp
