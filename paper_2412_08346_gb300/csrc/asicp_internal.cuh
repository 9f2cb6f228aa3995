// Internal declarations shared by the kernels and the C-ABI of libasicp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace asicp {

constexpr int kDeviceSlots = 64;       // devices a process can use the library on

// A launch value that depends on the device (its SM count, an occupancy) and
// sets the kernel attributes it relies on: compute() runs once per device, with
// that device current, under a lock, so several devices and several host
// threads each get their own value.  Returns 0 (an invalid grid, which the
// launch then reports) if the current device cannot be read.
template <class F>
int per_device_value(int (&cache)[kDeviceSlots], std::mutex &mu, F compute)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDeviceSlots) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) cache[dev] = compute();
    return cache[dev];
}

constexpr int kRefTilePts = 2048;      // object points per shared-memory tile of the matching kernel
constexpr int kFwdSums = 13;           // per-particle matching sums (see match kernel)
constexpr int kColSums = 22;           // per-particle collision sums (see collision kernel)
constexpr int kMaxK = 1024;            // particles per preshape (one update CTA per preshape)
constexpr int kMaxN = 6144;            // gripper points per preshape (reverse matching keeps 32 B per point in shared memory)

// error word written by device code (host reads it back after synchronising)
enum : int { kDevOk = 0, kDevNonFinite = 1, kDevTimeout = 2 };

struct SdfMeta {           // one preshape's grid
    const float *grid;     // nx*ny*nz values, x fastest, positive inside the gripper
    const float4 *cells;   // the same values corner-packed: per cell (x fastest over the
                           // (nx-1)(ny-1)(nz-1) cells) its 8 corners as two float4,
                           // {c000, c100, c010, c110} {c001, c101, c011, c111} (index x, y, z)
    int nx, ny, nz;
    float ox, oy, oz;      // position of node (0,0,0)
    float voxel;
    float lo[3], hi[3];    // box (gripper frame) holding every cell with a positive corner
};

// Rotation of a (unit) quaternion in the homogeneous form
// R = (w^2 - |v|^2) I + 2 v v^T + 2 w [v]_x, evaluated with explicit
// round-to-nearest operations so every kernel gets bit-identical matrices.
__device__ __forceinline__ void quat_rot_f32(float w, float x, float y, float z, float R[9])
{
    float a = __fsub_rn(__fmul_rn(w, w), __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    R[0] = __fadd_rn(a, __fmul_rn(2.f, xx));
    R[1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
    R[2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
    R[3] = __fmul_rn(2.f, __fadd_rn(xy, wz));
    R[4] = __fadd_rn(a, __fmul_rn(2.f, yy));
    R[5] = __fmul_rn(2.f, __fsub_rn(yz, wx));
    R[6] = __fmul_rn(2.f, __fsub_rn(xz, wy));
    R[7] = __fmul_rn(2.f, __fadd_rn(yz, wx));
    R[8] = __fadd_rn(a, __fmul_rn(2.f, zz));
}

__device__ __forceinline__ void quat_rot_f64(double w, double x, double y, double z, double R[9])
{
    double a = w * w - (x * x + y * y + z * z);
    R[0] = a + 2 * x * x;         R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);   R[4] = a + 2 * y * y;       R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);   R[7] = 2 * (y * z + w * x); R[8] = a + 2 * z * z;
}

// s' = R s + t in float32, fixed operation order (shared by every kernel that
// needs transformed gripper points, so forward and reverse matching agree).
__device__ __forceinline__ float3 xform_f32(const float R[9], float tx, float ty, float tz, float sx, float sy, float sz)
{
    float3 o;
    o.x = __fmaf_rn(R[0], sx, __fmaf_rn(R[1], sy, __fmaf_rn(R[2], sz, tx)));
    o.y = __fmaf_rn(R[3], sx, __fmaf_rn(R[4], sy, __fmaf_rn(R[5], sz, ty)));
    o.z = __fmaf_rn(R[6], sx, __fmaf_rn(R[7], sy, __fmaf_rn(R[8], sz, tz)));
    return o;
}

// Exact-form squared distance |a - b|^2 in float32, fixed order.
__device__ __forceinline__ float dist2_f32(float ax, float ay, float az, float bx, float by, float bz)
{
    float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Exact-form nearest point among object points [lo, hi) (index order, strict <).
__device__ __forceinline__ void exact_scan(const float4 *__restrict__ R, int lo, int hi, float sx, float sy, float sz,
                                           float &best, int &bi)
{
    for (int r = lo; r < hi; ++r) {
        const float4 v = __ldg(R + r);
        const float d = dist2_f32(sx, sy, sz, v.x, v.y, v.z);
        if (d < best) { best = d; bi = r; }
    }
}

// Exact-form nearest point of query (qx, qy, qz) among all M object points, found by
// the whole warp together (lane l takes points l, l + 32, ...; ties to the lower
// index); every lane receives the result.  Call with all 32 lanes.
__device__ __forceinline__ void warp_exact_all(const float4 *__restrict__ R, int M, float qx, float qy, float qz,
                                               float &best, int &bi)
{
    float wb = __int_as_float(0x7f800000);
    int wi = 0x7fffffff;
    for (int r = (int)(threadIdx.x & 31); r < M; r += 32) {
        const float4 v = __ldg(R + r);
        const float d = dist2_f32(qx, qy, qz, v.x, v.y, v.z);
        if (d < wb) { wb = d; wi = r; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, wb, off);
        const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
        if (ob < wb || (ob == wb && oi < wi)) { wb = ob; wi = oi; }
    }
    best = wb;
    bi = wi < M ? wi : 0;    // no finite distance at all (not reached with finite inputs)
}

// Double-float accumulation (hi + lo, ~48-bit significand) from float32 error-free
// transformations: products are split exactly by an FMA, sums by two-sum.  Used
// for the per-particle sums, where float64 arithmetic would dominate the run time
// on GB300 (float64 rate 1/64 of float32).
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void df_add(dfloat &x, float v)
{
    float s, e;
    two_sum(x.hi, v, s, e);
    x.hi = s;
    x.lo = __fadd_rn(x.lo, e);
}

__device__ __forceinline__ void df_add_prod(dfloat &x, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);      // a * b = p + pe exactly
    float s, e;
    two_sum(x.hi, p, s, e);
    x.hi = s;
    x.lo = __fadd_rn(x.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ void df_merge(dfloat &x, const dfloat &y)
{
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    x.hi = s;
    x.lo = __fadd_rn(x.lo, __fadd_rn(e, y.lo));
}

template <int N>
__device__ __forceinline__ void warp_sum_df(dfloat (&v)[N])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            dfloat y;
            y.hi = __shfl_xor_sync(0xffffffffu, v[c].hi, o);
            y.lo = __shfl_xor_sync(0xffffffffu, v[c].lo, o);
            df_merge(v[c], y);
        }
}

template <int N>
__device__ __forceinline__ void warp_sum_f64(double (&v)[N])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < N; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
}

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns the launch status.
// ---------------------------------------------------------------- layout
// Several objects can be optimised in one pass.  Particles are numbered object
// by object, preshape by preshape: group g = o * P + p holds the K_g particles
// grp_off[g] .. grp_off[g + 1] - 1 of preshape p on object o.
struct ObjMeta {
    const float4 *R;          // [M] object points
    const ulonglong2 *Rx;     // [Mpad] screening layout (pairs of (-2r, |r|^2)), Mpad = whole tiles
    const float *Rt;          // [Mpad / 128] augmented tiles of the tensor-core kernel (8 KB each)
    const float4 *C;          // [Mc] collision points (may alias R)
    int M, Mpad, Mc, chunks;  // chunks = ceil(Mc / kColChunk)
    int pfirst, np;           // first particle and number of particles of this object
    long long colidx_base;    // this object's collision lists start here ([np][Mc] ints)
    long long csum_base;      // this object's chunk sums start here ([np][chunks] slots)
};

struct Layout {
    int P, N, G, nobj, T;     // preshapes, gripper points, groups, objects, particles
    const int *part_grp;      // [T] group of every particle
    const int *grp_off;       // [G + 1] first particle of every group
    const ObjMeta *obj;       // [nobj]
    const double *com;        // [nobj][3] object centroids (CoM)
    const float4 *frame;      // [nobj] screening frame: centre c (x, y, z; the bounding-box
                              // centre) and w = max |fl(r - c)| rounded up (see ref_prep_kernel)
};

// A unit of forward-matching work: queries [q0, q0 + nq) of the flattened
// (particle, gripper point) space, all on object `obj` (nq <= 1024).
struct FwdItem {
    long long q0;
    int nq, obj;
};

struct FwdArgs {
    Layout L;
    const float4 *S;         // [P][N] gripper points (gripper frame)
    const float *theta;      // [T][8]
    const FwdItem *items;    // [n_items] work items (null: object 0, consecutive 1024-query items)
    const int *cta_off;      // [grid + 1]: CTA b runs items cta_off[b] .. cta_off[b+1]-1 (null: round-robin)
    int n_items;
    int *err;                // error word
    int *nn_idx;             // [T][N] nearest object point per query
    float *dbg_d2;           // [T][N] or null
    float *dbg_sp;           // [T][N][3] or null
    int4 *cand;              // [T][N] tensor-core shape only: candidate chunks per query
    int variant;             // kernel shape (0 .. kFwdVariants - 1), chosen by the autotuner
    int expire_test;         // float32 shapes: the first copy wait of a CTA waits on an mbarrier
                             // that nothing arrives at, for kTestWaitCycles (tests the timeout path)
};
constexpr int kFwdItemQueries = 1024;  // queries per forward-matching work item
constexpr int kFwdVariants = 8;        // kernel shapes of the forward matching (7: tensor cores)
cudaError_t launch_fwd_match(const FwdArgs &a, cudaStream_t st);
// The tensor-core shape leaves the exact choice to a second kernel (launch it after
// launch_fwd_match on the same stream); the float32 shapes make it themselves.
inline bool fwd_has_exact_kernel(int v) { return v == kFwdVariants - 1; }
cudaError_t launch_fwd_exact(const FwdArgs &a, cudaStream_t st);
int fwd_grid_size();                   // first call sets the kernels' attributes
int fwd_shape_grid(int v);             // CTAs of kernel shape v (a whole number per SM)
int fwd_shape_threads(int v);          // threads per CTA of kernel shape v
int fwd_shape_queries(int v);          // queries per work item (at most) of kernel shape v
const char *fwd_variant_name(int v);
cudaError_t init_collision_attributes();
cudaError_t init_update_attributes();
// Screening layout of R relative to the frame's centre.  compute_frame = true finds the
// centre and radius of R and stores them in *frame; false keeps the given frame (a
// subset of a cloud whose frame is already set, e.g. a mini-batch).
cudaError_t launch_ref_prep(const float4 *R, int M, int Mpad, void *Rx, float4 *frame, bool compute_frame,
                            cudaStream_t st);
cudaError_t launch_tc_ref_prep(const float4 *R, int M, int Mpad, const float4 *frame, void *Rt, cudaStream_t st);
size_t tc_ref_bytes(int Mpad);         // bytes of the tensor-core object tiles
cudaError_t launch_fwd_match_tc(const FwdArgs &a, cudaStream_t st);
cudaError_t launch_tc_exact(const FwdArgs &a, cudaStream_t st);
int fwd_tc_grid();
int fwd_tc_threads();

constexpr int kColChunk = 64;          // colliding points per reverse-matching work item

struct CollideArgs {
    Layout L;
    const float *theta;       // [T][8]
    const SdfMeta *meta;      // [P]
    const float4 *S;          // [P][N]
    const int *nn_idx;        // [T][N] forward correspondences
    int *ncol;                // [T]
    int *colidx;              // collision lists (see ObjMeta::colidx_base)
    double *fsums;            // [T][kFwdSums]
    double *csums;            // chunk sums (see ObjMeta::csum_base) [.][kColSums]
    int *dbg_colnn;           // like colidx, or null
    int *col_items;           // (count, next) of the reverse-matching work list
    int *col_list;            // [2 * items] (particle, chunk) pairs
    const int *err;           // error word: a kernel of the pass found an error, skip the work
};
cudaError_t launch_collide(const CollideArgs &a, cudaStream_t st);
cudaError_t launch_collide_nn(const CollideArgs &a, cudaStream_t st);

struct UpdateArgs {
    Layout L;
    float *theta;             // [T][8] in/out
    const double *fsums;      // [T][kFwdSums]
    const double *csums;      // chunk sums
    const int *ncol;          // [T]
    const double *pconst;     // [P][12]: sum s (3), sum s s^T (xx,xy,xz,yy,yz,zz), pad
    double w_com;
    int mode;                 // 0: evaluate only, 1: SVGD step, 2: SGD step
    float gamma, eta_svgd, eta_sgd;
    int bandwidth_mode;
    float h_fixed;
    float conv_tol;           // < 0 disables
    double *cost;             // [T]
    double *grad;             // [T][8]
    double *prev_cost;        // [T]
    int *frozen;              // [T]
    float *phi;               // [T][8]
    float *h;                 // [G]
    int *col_items;           // collision work-list counters (count, next), cleared for the next pass
    float prior_t_sigma;      // Gaussian prior on t around the object's CoM (<= 0: off)
    float prior_q_kappa;      // von Mises prior on q (<= 0: off)
    float prior_q_mean[4];    // its unit mean
    const int *err;           // error word: a kernel of the pass found an error, skip the work
};
cudaError_t launch_finalize(const UpdateArgs &a, cudaStream_t st);   // cost/gradient, convergence, SGD step
cudaError_t launch_stein(const UpdateArgs &a, cudaStream_t st);      // SVGD step (mode 1)

cudaError_t launch_pack_points(const float *xyz, int n, float4 *out, int *err, cudaStream_t st);
cudaError_t launch_check_finite(const float *v, long long n, int *err, cudaStream_t st);
cudaError_t launch_centroid(const float4 *X, int n, double *out3, cudaStream_t st);
cudaError_t launch_preshape_consts(const float4 *S, int N, double *out12, cudaStream_t st);
cudaError_t launch_fibonacci(const Layout &L, float radius, int mode, float *theta, cudaStream_t st);
cudaError_t launch_gather_points(const float4 *R, const int *idx, int n, float4 *out, cudaStream_t st);
cudaError_t launch_store_meta(ObjMeta *dst, const ObjMeta &v, cudaStream_t st);
cudaError_t launch_set_theta(const float *theta7, int T, float *theta8, int *err, cudaStream_t st);
cudaError_t launch_sdf_box(const float *grid, int nx, int ny, int nz, int *box6, cudaStream_t st);
cudaError_t launch_sdf_pack_cells(const float *grid, int nx, int ny, int nz, float4 *cells, cudaStream_t st);
size_t sdf_cells_bytes(int nx, int ny, int nz);
cudaError_t launch_select(const Layout &L, const double *cost, const int *ncol, int *order, cudaStream_t st);
cudaError_t launch_uniform_groups(int *part_grp, int *grp_off, int P, int K, cudaStream_t st);

}  // namespace asicp
