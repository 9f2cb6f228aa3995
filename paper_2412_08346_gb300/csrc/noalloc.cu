// asicp_match_noalloc: forward matching (nearest object point for every
// particle and gripper point) for callers that must not allocate device memory.
//
// Who cannot allocate: real-time control loops that have reserved their memory
// at start-up and must not stall (cudaMalloc / cudaFree can synchronise the
// device and take milliseconds), runtimes that hand out all device memory from
// their own pre-sized pool and forbid libraries from going around it, and code
// that runs while another component has the device memory budget pinned.  For
// them this entry point keeps all of its scratch in one file-scope device array
// of fixed size, so it never calls cudaMalloc, cudaFree or an allocating
// library routine.
//
// The array lives in every GPU that loads the library until the process exits.
// Host code cannot use the array's name as a device address (in host code it is
// only a stand-in symbol), so on the first call on each device, with that device
// current, the address is fetched once with cudaGetSymbolAddress and cached;
// make that first call before any stream capture.  Every call on a device uses
// the same array and leaves its contents behind: calls that overlap on the GPU
// (other streams, other host threads) race, so callers must order them.
#include "../../include/asicp.h"
#include "asicp_internal.cuh"

#include <mutex>

namespace asicp {

namespace {

constexpr size_t kScratchBytes = 5u << 20;          // 5 MiB
constexpr int kMaxDevices = 64;

// Scratch layout (offsets in bytes, all 256-aligned):
//   poses     [ASICP_NOALLOC_MAX_PK][8] float     512 KiB
//   gripper   [ASICP_NOALLOC_MAX_PN] float4        1 MiB
//   object    [ASICP_NOALLOC_MAX_M] float4         1 MiB
//   screening [ASICP_NOALLOC_MAX_M] 16 B           1 MiB
//   staging   3 * max(M, P*N, 7/3 P*K) floats     768 KiB
//   particle -> preshape map [P*K] int, preshape offsets [P+1] int   64 KiB each
//   object table, screening frame (float4), error word (int)
constexpr size_t kOffPoses = 0;
constexpr size_t kOffGripper = kOffPoses + (size_t)ASICP_NOALLOC_MAX_PK * 8 * 4;
constexpr size_t kOffObject = kOffGripper + (size_t)ASICP_NOALLOC_MAX_PN * 16;
constexpr size_t kOffScreen = kOffObject + (size_t)ASICP_NOALLOC_MAX_M * 16;
constexpr size_t kOffStage = kOffScreen + (size_t)ASICP_NOALLOC_MAX_M * 16;
constexpr size_t kStageFloats = 3 * (size_t)ASICP_NOALLOC_MAX_M;
constexpr size_t kOffPartGrp = kOffStage + kStageFloats * 4;
constexpr size_t kOffGrpOff = kOffPartGrp + (size_t)ASICP_NOALLOC_MAX_PK * 4;
constexpr size_t kOffObjMeta = kOffGrpOff + ((size_t)ASICP_NOALLOC_MAX_PK + 64) * 4;
constexpr size_t kOffFrame = kOffObjMeta + 256;
constexpr size_t kOffErr = kOffFrame + 256;
static_assert(sizeof(ObjMeta) <= 256, "object table slot too small");
static_assert(kOffErr + 256 <= kScratchBytes, "scratch layout exceeds the static array");
static_assert(kStageFloats >= 3 * (size_t)ASICP_NOALLOC_MAX_PN && kStageFloats >= 7 * (size_t)ASICP_NOALLOC_MAX_PK,
              "staging area too small");

__device__ __align__(256) unsigned char g_match_scratch[kScratchBytes];

unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_match_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool device_accessible(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace asicp

using namespace asicp;

extern "C" asicp_status asicp_match_noalloc(const float *theta, int P, int K, const float *S_xyz, int N,
                                            const float *R_xyz, int M, int *nn_idx, void *cuda_stream)
{
    if (!theta || !S_xyz || !R_xyz || !nn_idx || P < 1 || K < 1 || N < 1 || M < 1) return ASICP_ERR_INVALID_ARG;
    if ((long long)P * K > ASICP_NOALLOC_MAX_PK || (long long)P * N > ASICP_NOALLOC_MAX_PN ||
        M > ASICP_NOALLOC_MAX_M)
        return ASICP_ERR_INVALID_ARG;     // beyond the fixed scratch: use the context API instead
    if (!device_accessible(nn_idx)) return ASICP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) return ASICP_ERR_CUDA;

    float *poses = reinterpret_cast<float *>(base + kOffPoses);
    float4 *grip = reinterpret_cast<float4 *>(base + kOffGripper);
    float4 *obj = reinterpret_cast<float4 *>(base + kOffObject);
    ulonglong2 *screen = reinterpret_cast<ulonglong2 *>(base + kOffScreen);
    float *stage = reinterpret_cast<float *>(base + kOffStage);
    float4 *frame = reinterpret_cast<float4 *>(base + kOffFrame);
    int *err = reinterpret_cast<int *>(base + kOffErr);
    int *part_grp = reinterpret_cast<int *>(base + kOffPartGrp);
    int *grp_off = reinterpret_cast<int *>(base + kOffGrpOff);
    ObjMeta *objmeta = reinterpret_cast<ObjMeta *>(base + kOffObjMeta);
    const int PK = P * K;
    const int Mpad = (M + kRefTilePts - 1) / kRefTilePts * kRefTilePts;

#define NOALLOC_CK(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return ASICP_ERR_CUDA; } } while (0)
    NOALLOC_CK(cudaMemsetAsync(err, 0, sizeof(int), st));   // the array keeps the last call's error word
    // inputs that are host memory go through the staging area (a copy, not an allocation)
    auto src = [&](const float *p, size_t n) -> const float * {
        if (device_accessible(p)) return p;
        if (cudaMemcpyAsync(stage, p, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
        return stage;
    };
    const float *th = src(theta, (size_t)PK * 7);
    if (!th) return ASICP_ERR_CUDA;
    NOALLOC_CK(launch_set_theta(th, PK, poses, err, st));
    const float *sx = src(S_xyz, (size_t)P * N * 3);
    if (!sx) return ASICP_ERR_CUDA;
    NOALLOC_CK(launch_pack_points(sx, P * N, grip, err, st));
    const float *rx = src(R_xyz, (size_t)M * 3);
    if (!rx) return ASICP_ERR_CUDA;
    NOALLOC_CK(launch_pack_points(rx, M, obj, err, st));
    NOALLOC_CK(launch_ref_prep(obj, M, Mpad, screen, frame, true, st));
    NOALLOC_CK(launch_uniform_groups(part_grp, grp_off, P, K, st));
    // a non-finite input stops the call before the matching: nn_idx stays untouched
    NOALLOC_CK(cudaStreamSynchronize(st));
    int e_in = 0;
    NOALLOC_CK(cudaMemcpy(&e_in, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e_in == kDevNonFinite) return ASICP_ERR_INVALID_ARG;
    ObjMeta om{};          // one object holding every particle (copied by value below)
    om.R = obj;
    om.Rx = screen;
    om.C = obj;
    om.M = M; om.Mpad = Mpad; om.Mc = M; om.chunks = 0;
    om.pfirst = 0; om.np = PK;
    NOALLOC_CK(cudaMemcpyAsync(objmeta, &om, sizeof(ObjMeta), cudaMemcpyHostToDevice, st));

    FwdArgs fa{};
    fa.L.P = P; fa.L.N = N; fa.L.G = P; fa.L.nobj = 1; fa.L.T = PK;
    fa.L.part_grp = part_grp;
    fa.L.grp_off = grp_off;
    fa.L.obj = objmeta;
    fa.L.com = nullptr;
    fa.L.frame = frame;
    fa.S = grip;
    fa.theta = poses;
    fa.items = nullptr;    // consecutive work items of object 0
    fa.n_items = (int)(((long long)PK * N + kFwdItemQueries - 1) / kFwdItemQueries);
    fa.err = err;
    fa.nn_idx = nn_idx;
    NOALLOC_CK(launch_fwd_match(fa, st));
    NOALLOC_CK(cudaStreamSynchronize(st));   // also keeps `om` alive until its copy is done
    int e = 0;
    NOALLOC_CK(cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost));
#undef NOALLOC_CK
    if (e == kDevNonFinite) return ASICP_ERR_INVALID_ARG;
    if (e == kDevTimeout) return ASICP_ERR_TIMEOUT;
    return ASICP_OK;
}
