// Per-particle cost and gradient, Stein direction and the particle update
// (Eqs. 3, 7-11, 13-18), plus the small set-up kernels (packing, centroids,
// Fibonacci initial poses, ranking).
#include "asicp_internal.cuh"

namespace asicp {

namespace {

// Quaternion gradient g_k = sum_ab (dR_ab/dq_k) E_ab for the homogeneous form
// R = (w^2 - |v|^2) I + 2 v v^T + 2 w [v]_x, with E = sum_i e_i s_i^T:
//   dR/dw   = 2 w I + 2 [v]_x
//   dR/dv_k = -2 v_k I + 2 (e_k v^T + v e_k^T) + 2 w [e_k]_x
// This equals sum_i J(s_i)^T e_i, the rotation gradient of Eqs. 5 and 17.
__device__ void quat_grad_from_E(const double q[4], const double E[9], double g[4])
{
    const double w = q[0], v[3] = {q[1], q[2], q[3]};
    const double tr = E[0] + E[4] + E[8];
    const double kx = E[7] - E[5], ky = E[2] - E[6], kz = E[3] - E[1];   // <[e_k]_x, E>
    g[0] = 2 * w * tr + 2 * (v[0] * kx + v[1] * ky + v[2] * kz);
    const double ks[3] = {kx, ky, kz};
    for (int k = 0; k < 3; ++k) {
        double rowv = E[k * 3 + 0] * v[0] + E[k * 3 + 1] * v[1] + E[k * 3 + 2] * v[2];
        double colv = E[0 * 3 + k] * v[0] + E[1 * 3 + k] * v[1] + E[2 * 3 + k] * v[2];
        g[1 + k] = -2 * v[k] * tr + 2 * rowv + 2 * colv + 2 * w * ks[k];
    }
}

// sum_i |R s_i + t - x_i|^2, sum_i (R s_i + t - x_i) and sum_i (R s_i + t - x_i) s_i^T
// from the linear sums: ss = sum s (3), SS = sum s s^T (9, full), xs = sum x,
// XS = sum x s^T (9), xx = sum |x|^2, n terms.
__device__ void residual_moments(const double R[9], const double t[3], double n, const double ss[3],
                                 const double SS[9], const double xs[3], const double XS[9], double xx,
                                 double *se2, double Se[3], double E[9])
{
    double Rs[3];
    for (int a = 0; a < 3; ++a) Rs[a] = R[a * 3 + 0] * ss[0] + R[a * 3 + 1] * ss[1] + R[a * 3 + 2] * ss[2];
    // R is the homogeneous form of the quaternion's rotation (|q|^2 times a rotation), so
    // R^T R = |q|^4 I and sum_i |R s_i|^2 = |q|^4 tr(SS); |q|^4 is the squared norm of a column
    const double q4 = R[0] * R[0] + R[3] * R[3] + R[6] * R[6];
    const double quad = q4 * (SS[0] + SS[4] + SS[8]);
    double cross = 0.0;
    for (int a = 0; a < 9; ++a) cross += R[a] * XS[a];
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double tRs = t[0] * Rs[0] + t[1] * Rs[1] + t[2] * Rs[2];
    const double tx = t[0] * xs[0] + t[1] * xs[1] + t[2] * xs[2];
    *se2 = quad + n * tt + xx + 2 * tRs - 2 * tx - 2 * cross;
    for (int a = 0; a < 3; ++a) Se[a] = Rs[a] + n * t[a] - xs[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            E[a * 3 + b] = R[a * 3 + 0] * SS[0 * 3 + b] + R[a * 3 + 1] * SS[1 * 3 + b] + R[a * 3 + 2] * SS[2 * 3 + b] +
                           t[a] * ss[b] - XS[a * 3 + b];
}

__device__ __forceinline__ void sym_full(const double *s6, double S[9])
{
    S[0] = s6[0]; S[1] = s6[1]; S[2] = s6[2];
    S[3] = s6[1]; S[4] = s6[3]; S[5] = s6[4];
    S[6] = s6[2]; S[7] = s6[4]; S[8] = s6[5];
}

__device__ __forceinline__ float pair_d2(float4 a, float4 b)
{
    return dist2_f32(a.x, a.y, a.z, b.x, b.y, b.z);
}

}  // namespace

// Per particle (one thread each, small CTAs so the float64 work spreads over
// many SMs):
//  1. cost and gradient from the matching sums (Eqs. 13-17) or, for a particle
//     with colliding points, from the collision sums (Eq. 18 with Eqs. 4-5),
//     quaternion block projected onto the tangent space at q;
//  2. convergence bookkeeping (SGD phase);
//  3. mode 2: the SGD-ICP update of Eq. 3 (A = I); modes 0 (evaluate only) and 1
//     (SVGD, done by stein_kernel) leave the poses alone.
//  Thread 0 of CTA 0 also clears the collision work-list counters for the next pass.
constexpr int kFinalizeThreads = 4;      // 192 CTAs for 768 particles: float64 chains spread over every SM

__global__ void __launch_bounds__(kFinalizeThreads) finalize_kernel(const UpdateArgs a)
{
    if (a.err && *a.err != kDevOk) return;    // an earlier kernel of the pass gave up: its sums are not valid
    const int pk = blockIdx.x * blockDim.x + threadIdx.x;
    if (pk == 0 && a.col_items) { a.col_items[0] = 0; a.col_items[1] = 0; }
    if (pk >= a.L.T) return;
    const int grp = a.L.part_grp[pk], p = grp % a.L.P, o = grp / a.L.P;
    const int N = a.L.N;
    double t[3], q[4], g[7];
    const float *th = a.theta + (size_t)pk * 8;
    for (int c = 0; c < 3; ++c) t[c] = th[c];
    for (int c = 0; c < 4; ++c) q[c] = th[3 + c];
    double R[9];
    quat_rot_f64(q[0], q[1], q[2], q[3], R);
    const int nc = a.ncol[pk];
    double se2, Se[3], E[9], cnt;
    if (nc == 0) {
        double fs[kFwdSums];
        for (int c = 0; c < kFwdSums; ++c) fs[c] = a.fsums[(size_t)pk * kFwdSums + c];
        const double *pc = a.pconst + (size_t)p * 12;
        double SS[9];
        sym_full(pc + 3, SS);
        residual_moments(R, t, (double)N, pc, SS, fs, fs + 3, fs[12], &se2, Se, E);
        // TCP-CoM term (Eq. 15) inside the 1/N, weight w_com (Eqs. 16-17)
        const double tcp[3] = {pc[0] / N, pc[1] / N, pc[2] / N};
        const double *com = a.L.com + 3 * o;
        double ec[3];
        for (int u = 0; u < 3; ++u)
            ec[u] = R[u * 3 + 0] * tcp[0] + R[u * 3 + 1] * tcp[1] + R[u * 3 + 2] * tcp[2] + t[u] - com[u];
        se2 += a.w_com * (ec[0] * ec[0] + ec[1] * ec[1] + ec[2] * ec[2]);
        for (int u = 0; u < 3; ++u) {
            Se[u] += a.w_com * ec[u];
            for (int v = 0; v < 3; ++v) E[u * 3 + v] += a.w_com * ec[u] * tcp[v];
        }
        cnt = (double)N;
    } else {
        // add the per-chunk collision sums in chunk order
        const ObjMeta &om = a.L.obj[o];
        const int used = (nc + kColChunk - 1) / kColChunk;
        const double *csp = a.csums + (om.csum_base + (long long)(pk - om.pfirst) * om.chunks) * kColSums;
        double cs[kColSums];
        for (int c = 0; c < kColSums; ++c) cs[c] = 0.0;
        for (int b = 0; b < used; ++b)
            for (int c = 0; c < kColSums; ++c) cs[c] += csp[(size_t)b * kColSums + c];
        double SS[9];
        sym_full(cs + 3, SS);
        residual_moments(R, t, (double)nc, cs, SS, cs + 9, cs + 12, cs[21], &se2, Se, E);
        cnt = (double)nc;
    }
    double gq[4];
    quat_grad_from_E(q, E, gq);
    const double inv = 1.0 / cnt;
    for (int u = 0; u < 3; ++u) g[u] = Se[u] * inv;
    for (int u = 0; u < 4; ++u) gq[u] *= inv;
    const double dq = gq[0] * q[0] + gq[1] * q[1] + gq[2] * q[2] + gq[3] * q[3];
    for (int u = 0; u < 4; ++u) g[3 + u] = gq[u] - dq * q[u];
    const double cost = se2 * inv;
    a.cost[pk] = cost;
    for (int u = 0; u < 7; ++u) a.grad[(size_t)pk * 8 + u] = g[u];
    int frozen = a.frozen[pk];
    if (a.mode == 2 && a.conv_tol >= 0.f) {
        const double prev = a.prev_cost[pk];
        if (nc > 0) frozen = 0;
        else if (prev >= 0.0 && fabs(cost - prev) <= (double)a.conv_tol * prev) frozen = 1;
        a.frozen[pk] = frozen;
    }
    if (a.mode != 0) a.prev_cost[pk] = cost;
    if (a.mode == 2) {
        float *tw = a.theta + (size_t)pk * 8;
        for (int u = 0; u < 7; ++u) a.phi[(size_t)pk * 8 + u] = 0.f;
        if (pk < a.L.G) a.h[pk] = 0.f;
        if (!frozen) {
            double nq[4];
            for (int u = 0; u < 4; ++u) nq[u] = q[u] - (double)a.eta_sgd * g[3 + u];
            const double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
            for (int u = 0; u < 3; ++u) tw[u] = (float)(t[u] - (double)a.eta_sgd * g[u]);
            for (int u = 0; u < 4; ++u) tw[3 + u] = (float)(nq[u] / nn);
        }
    }
}

// SVGD phase, kSteinSplit CTAs of kSteinThreads per preshape.  Every CTA of a
// preshape computes the bandwidth (the same deterministic selection), then the
// Stein direction of its share of ceil(K / kSteinSplit) particles; the poses are
// updated by stein_update_kernel afterwards, because every CTA reads all poses of
// its preshape.  For the bandwidth each particle i is served by T = kSteinThreads
// / K' threads (K' = K rounded up to a power of two); for the direction each
// particle of the share by T' = kSteinThreads / K'' threads (K'' = the share
// rounded up), at most a warp:
//  - bandwidth: exact lower median of |t_i - t_j|^2 (i < j): the value range is
//    narrowed by histograms over linear bins (usually one pass) until the bin
//    holding the median has at most kSelCand values, which are then ranked
//    exactly; every unordered pair is visited once per pass (thread (i, sub)
//    takes partners i + o (mod K), o = 1 + sub + T m <= K/2, the o = K/2 pairs
//    only from i < K/2 when K is even);
//  - Stein direction of Eq. 8 read as the mean of Eq. 6 with the kernels of
//    Eqs. 9-10 per block: thread (i, sub) sums over j = sub, sub + T', ..., the T'
//    partial sums of particle i (adjacent lanes) are added by shuffles, and
//    written to phi;
//  - the update of Eq. 7 (stein_update_kernel).
constexpr int kSteinThreads = 1024;
constexpr int kSteinSplit = 8;         // CTAs per preshape
constexpr int kSelBins = 1024;         // histogram bins per narrowing pass of the median selection
constexpr int kSelCand = 1024;         // values ranked exactly at the end

__global__ void __launch_bounds__(kSteinThreads) stein_kernel(const UpdateArgs a)
{
    if (a.err && *a.err != kDevOk) return;
    extern __shared__ float4 sm[];
    float4 *sT = sm;                  // [K] t (xyz)
    float4 *sQ = sm + kMaxK;          // [K] q (wxyz)
    float4 *sDt = sm + 2 * kMaxK;     // [K] -gamma N g_t
    float4 *sDq = sm + 3 * kMaxK;     // [K] -gamma N g_q
    __shared__ unsigned hist[kSelBins];
    __shared__ float cand[kSelCand];
    __shared__ unsigned s_wsum[kSteinThreads / 32];
    __shared__ unsigned s_lo, s_hi, s_rank, s_n, s_bin, s_before, s_fill;
    __shared__ float s_h;

    const int grp = blockIdx.x / kSteinSplit, part = blockIdx.x % kSteinSplit;
    const int base = a.L.grp_off[grp], K = a.L.grp_off[grp + 1] - base;
    const int share = (K + kSteinSplit - 1) / kSteinSplit, i0 = part * share;
    if (K <= 0 || i0 >= K) return;      // (whole CTAs; no CTA waits on another)
    int Kp = 1;
    while (Kp < K) Kp <<= 1;
    const int T = min(kSteinThreads / Kp, 32);        // threads per particle: a power of two <= a warp
    const int i = threadIdx.x / T, sub = threadIdx.x % T;
    const bool active = i < K;
    const float gN = -a.gamma * (float)a.L.N;
    const double *com = a.L.com + 3 * (grp / a.L.P);
    const float cx = (float)com[0], cy = (float)com[1], cz = (float)com[2];
    const float pt = a.prior_t_sigma > 0.f ? -a.gamma / (a.prior_t_sigma * a.prior_t_sigma) : 0.f;
    const float pq = a.prior_q_kappa > 0.f ? a.gamma * a.prior_q_kappa : 0.f;
    const float *mu = a.prior_q_mean;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        const size_t pj = (size_t)base + j;
        const float *th = a.theta + pj * 8;
        const double *g = a.grad + pj * 8;
        sT[j] = make_float4(th[0], th[1], th[2], 0.f);
        sQ[j] = make_float4(th[3], th[4], th[5], th[6]);
        // drive gamma (-N g + grad log p): Gaussian prior on t, von Mises on q (both off at 0)
        const float m = mu[0] * th[3] + mu[1] * th[4] + mu[2] * th[5] + mu[3] * th[6];
        const float sq = m < 0.f ? -pq : pq;
        sDt[j] = make_float4(gN * (float)g[0] + pt * (th[0] - cx), gN * (float)g[1] + pt * (th[1] - cy),
                             gN * (float)g[2] + pt * (th[2] - cz), 0.f);
        sDq[j] = make_float4(gN * (float)g[3] + sq * mu[0], gN * (float)g[4] + sq * mu[1],
                             gN * (float)g[5] + sq * mu[2], gN * (float)g[6] + sq * mu[3]);
    }
    __syncthreads();

    float h;
    if (a.bandwidth_mode == 1) {
        h = a.h_fixed;
    } else if (K < 2) {
        h = 1.f;
    } else {
        const unsigned long long L = (unsigned long long)K * (K - 1) / 2;
        const int half = K / 2;
        const int trips = (half + T - 1) / T;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const float4 ti = sT[active ? i : 0];
        // squared distance of this thread's m-th pair, or -1 when it has none
        auto pair_at = [&](int m) -> float {
            const int o = 1 + sub + T * m;
            int jj = i + o;
            jj -= jj >= K ? K : 0;
            const bool valid = active && o <= half && !((K & 1) == 0 && o == half && i >= half);
            return valid ? pair_d2(ti, sT[jj]) : -1.f;
        };
        // range of all pair values (non-negative floats order like their bit patterns)
        unsigned vmin = 0xffffffffu, vmax = 0u;
        for (int m = 0; m < trips; ++m) {
            const float v = pair_at(m);
            if (v >= 0.f) { vmin = min(vmin, __float_as_uint(v)); vmax = max(vmax, __float_as_uint(v)); }
        }
        vmin = __reduce_min_sync(0xffffffffu, vmin);
        vmax = __reduce_max_sync(0xffffffffu, vmax);
        if (threadIdx.x == 0) { s_lo = 0xffffffffu; s_hi = 0u; s_rank = (unsigned)((L - 1) / 2); }
        __syncthreads();
        if (lane == 0) { atomicMin(&s_lo, vmin); atomicMax(&s_hi, vmax); }
        __syncthreads();
        // narrow [lo, hi] (it holds the answer, with s_rank values of the set below lo)
        // by histograms over kSelBins linear bins until the bin holding the answer has at
        // most kSelCand values, then rank those exactly; binning is monotone in the value,
        // so a bin holds a contiguous run of the sorted values
        float med = 0.f;
        for (int pass = 0;; ++pass) {
            const float lo = __uint_as_float(s_lo), hi = __uint_as_float(s_hi);
            if (!(lo < hi) || pass == 32) { med = lo; break; }   // (32: not reached with finite values)
            const float scale = (float)kSelBins / (hi - lo);
            auto bin_of = [&](float v) { return min(kSelBins - 1, (int)((v - lo) * scale)); };
            for (int b = threadIdx.x; b < kSelBins; b += blockDim.x) hist[b] = 0u;
            __syncthreads();
            for (int m = 0; m < trips; ++m) {
                const float v = pair_at(m);
                if (v >= lo && v <= hi) atomicAdd(&hist[bin_of(v)], 1u);
            }
            __syncthreads();
            // exclusive scan over the bins (one bin per thread), then the bin holding rank s_rank
            const int b = threadIdx.x;
            const unsigned cnt = b < kSelBins ? hist[b] : 0u;
            unsigned inc = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_wsum[warp] = inc;
            __syncthreads();
            unsigned before = inc - cnt;
            for (int w = 0; w < warp; ++w) before += s_wsum[w];
            const unsigned rank = s_rank;
            if (b < kSelBins && cnt > 0 && before <= rank && rank < before + cnt) {
                s_bin = (unsigned)b;
                s_before = before;
                s_n = cnt;
                s_fill = 0u;
                s_lo = 0xffffffffu;
                s_hi = 0u;
            }
            __syncthreads();
            const int bsel = (int)s_bin;
            const unsigned n = s_n;
            if (n <= (unsigned)kSelCand) {
                // gather the bin's values and rank them exactly
                for (int m = 0; m < trips; ++m) {
                    const float v = pair_at(m);
                    if (v >= lo && v <= hi && bin_of(v) == bsel) cand[atomicAdd(&s_fill, 1u)] = v;
                }
                __syncthreads();
                const unsigned r = s_rank - s_before;
                for (unsigned c = threadIdx.x; c < n; c += blockDim.x) {
                    const float v = cand[c];
                    unsigned less = 0u, equal = 0u;
                    for (unsigned e = 0; e < n; ++e) {
                        less += cand[e] < v;
                        equal += cand[e] == v;
                    }
                    if (less <= r && r < less + equal) s_lo = __float_as_uint(v);
                }
                __syncthreads();
                med = __uint_as_float(s_lo);
                break;
            }
            // too many: the bin's own value range becomes the new [lo, hi]
            unsigned bmin = 0xffffffffu, bmax = 0u;
            for (int m = 0; m < trips; ++m) {
                const float v = pair_at(m);
                if (v >= lo && v <= hi && bin_of(v) == bsel) {
                    bmin = min(bmin, __float_as_uint(v));
                    bmax = max(bmax, __float_as_uint(v));
                }
            }
            bmin = __reduce_min_sync(0xffffffffu, bmin);
            bmax = __reduce_max_sync(0xffffffffu, bmax);
            if (lane == 0) { atomicMin(&s_lo, bmin); atomicMax(&s_hi, bmax); }
            if (threadIdx.x == 0) s_rank -= s_before;
            __syncthreads();
        }
        if (threadIdx.x == 0) {     // float64 division and logarithm once, not per thread
            s_h = fmaxf((float)((double)med / log((double)K)), 1e-12f);
        }
        __syncthreads();
        h = s_h;
    }
    if (part == 0 && threadIdx.x == 0) a.h[grp] = h;

    // Stein direction of particles [i0, min(K, i0 + share)) of this preshape
    int Sp = 1;
    while (Sp < share) Sp <<= 1;
    const int T2 = min(kSteinThreads / Sp, 32);
    const int i2 = i0 + threadIdx.x / T2, sub2 = threadIdx.x % T2;
    const bool active2 = threadIdx.x / T2 < share && i2 < K;
    const float4 ti = sT[active2 ? i2 : 0], qi = sQ[active2 ? i2 : 0];
    const float inv_h = 1.f / h, two_h = 2.f / h;
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};     // t (3), q (4), sign count
    if (active2) {
        for (int jj = sub2; jj < K; jj += T2) {
            const float4 tj = sT[jj], qj = sQ[jj], dt = sDt[jj], dq = sDq[jj];
            const float ex = ti.x - tj.x, ey = ti.y - tj.y, ez = ti.z - tj.z;
            const float kt = expf(-(ex * ex + ey * ey + ez * ez) * inv_h);
            f[0] += kt * (dt.x + two_h * ex);
            f[1] += kt * (dt.y + two_h * ey);
            f[2] += kt * (dt.z + two_h * ez);
            const float c = qj.x * qi.x + qj.y * qi.y + qj.z * qi.z + qj.w * qi.w;
            f[3] += c * dq.x; f[4] += c * dq.y; f[5] += c * dq.z; f[6] += c * dq.w;
            f[7] += c < 0.f ? -1.f : 1.f;
        }
    }
    // the T2 threads of a particle are adjacent lanes of one warp (T2 is a power of two <= 32)
    for (int o = 1; o < T2; o <<= 1)
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u] += __shfl_xor_sync(0xffffffffu, f[u], o);
    if (active2 && sub2 == 0) {
        const size_t pk = (size_t)base + i2;
        const float invK = 1.f / (float)K;
        float g[7] = {f[0] * invK, f[1] * invK, f[2] * invK,
                      (f[3] + f[7] * qi.x) * invK, (f[4] + f[7] * qi.y) * invK,
                      (f[5] + f[7] * qi.z) * invK, (f[6] + f[7] * qi.w) * invK};
        // tangent projection at q_i (removes the radial kernel-gradient term)
        const float d = g[3] * qi.x + g[4] * qi.y + g[5] * qi.z + g[6] * qi.w;
        g[3] -= d * qi.x; g[4] -= d * qi.y; g[5] -= d * qi.z; g[6] -= d * qi.w;
        for (int u = 0; u < 7; ++u) a.phi[pk * 8 + u] = g[u];
    }
}

// The SVGD update of Eq. 7 from the Stein direction: t += eta phi_t, q <-
// normalise(q + eta phi_q) (phi_q is tangent at q), one thread per particle.
__global__ void stein_update_kernel(const UpdateArgs a)
{
    if (a.err && *a.err != kDevOk) return;
    const int pk = blockIdx.x * blockDim.x + threadIdx.x;
    if (pk >= a.L.T) return;
    float *th = a.theta + (size_t)pk * 8;
    const float *g = a.phi + (size_t)pk * 8;
    const float tx = th[0], ty = th[1], tz = th[2], qw = th[3], qx = th[4], qy = th[5], qz = th[6];
    const double es = a.eta_svgd;
    double nq[4] = {qw + es * g[3], qx + es * g[4], qy + es * g[5], qz + es * g[6]};
    const double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    th[0] = (float)(tx + es * g[0]);
    th[1] = (float)(ty + es * g[1]);
    th[2] = (float)(tz + es * g[2]);
    for (int u = 0; u < 4; ++u) th[3 + u] = (float)(nq[u] / nn);
}

cudaError_t init_update_attributes()
{
    return cudaFuncSetAttribute(stein_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float4) * 4 * kMaxK));
}

cudaError_t launch_finalize(const UpdateArgs &a, cudaStream_t st)
{
    finalize_kernel<<<(a.L.T + kFinalizeThreads - 1) / kFinalizeThreads, kFinalizeThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stein(const UpdateArgs &a, cudaStream_t st)
{
    const size_t smem = sizeof(float4) * 4 * (size_t)kMaxK;
    stein_kernel<<<a.L.G * kSteinSplit, kSteinThreads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stein_update_kernel<<<(a.L.T + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ set-up kernels
__global__ void pack_points_kernel(const float *xyz, int n, float4 *out, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = xyz[3 * (size_t)i], y = xyz[3 * (size_t)i + 1], z = xyz[3 * (size_t)i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicExch(err, kDevNonFinite);
    out[i] = make_float4(x, y, z, 0.f);
}

cudaError_t launch_pack_points(const float *xyz, int n, float4 *out, int *err, cudaStream_t st)
{
    pack_points_kernel<<<(n + 255) / 256, 256, 0, st>>>(xyz, n, out, err);
    return cudaGetLastError();
}

__global__ void check_finite_kernel(const float *v, long long n, int *err)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicExch(err, kDevNonFinite);
}

cudaError_t launch_check_finite(const float *v, long long n, int *err, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<(int)blocks, 256, 0, st>>>(v, n, err);
    return cudaGetLastError();
}

// Deterministic single-CTA float64 reductions (fixed thread striding + fixed tree).
template <int NV, class F>
__device__ void block_sum_f64(int n, F term, double *out)
{
    __shared__ double red[32][NV];
    double acc[NV];
    for (int c = 0; c < NV; ++c) acc[c] = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) term(i, acc);
    warp_sum_f64(acc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int c = 0; c < NV; ++c) red[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

__global__ void centroid_kernel(const float4 *X, int n, double *out3)
{
    __shared__ double tmp[3];
    block_sum_f64<3>(n, [&](int i, double *acc) {
        const float4 x = X[i];
        acc[0] += x.x; acc[1] += x.y; acc[2] += x.z;
    }, tmp);
    __syncthreads();
    if (threadIdx.x < 3) out3[threadIdx.x] = tmp[threadIdx.x] / n;
}

cudaError_t launch_centroid(const float4 *X, int n, double *out3, cudaStream_t st)
{
    centroid_kernel<<<1, 1024, 0, st>>>(X, n, out3);
    return cudaGetLastError();
}

__global__ void preshape_consts_kernel(const float4 *S, int N, double *out12)
{
    __shared__ double tmp[9];
    block_sum_f64<9>(N, [&](int i, double *acc) {
        const float4 s = S[i];
        const double x = s.x, y = s.y, z = s.z;
        acc[0] += x; acc[1] += y; acc[2] += z;
        acc[3] = fma(x, x, acc[3]); acc[4] = fma(x, y, acc[4]); acc[5] = fma(x, z, acc[5]);
        acc[6] = fma(y, y, acc[6]); acc[7] = fma(y, z, acc[7]); acc[8] = fma(z, z, acc[8]);
    }, tmp);
    __syncthreads();
    if (threadIdx.x < 9) out12[threadIdx.x] = tmp[threadIdx.x];
    if (threadIdx.x >= 9 && threadIdx.x < 12) out12[threadIdx.x] = 0.0;
}

cudaError_t launch_preshape_consts(const float4 *S, int N, double *out12, cudaStream_t st)
{
    preshape_consts_kernel<<<1, 1024, 0, st>>>(S, N, out12);
    return cudaGetLastError();
}

// Fibonacci sphere of K directions around the CoM (Section V); the same set for
// every preshape.  u_j: z = 1 - (2j+1)/K, azimuth j * pi * (3 - sqrt 5);
// t_j = CoM + radius u_j; q_j the smallest rotation taking +z (the approach
// axis) to -u_j, pi about x when -u_j = -z.  mode 1: the quarter-sphere lattice
// facing +x (upper half) plus min(6, K) poses above the object (see asicp.h).
__global__ void fibonacci_kernel(const Layout L, float radius, int mode, float *theta)
{
    const int pk = blockIdx.x * blockDim.x + threadIdx.x;
    if (pk >= L.T) return;
    const int grp = L.part_grp[pk];
    const int j = pk - L.grp_off[grp], K = L.grp_off[grp + 1] - L.grp_off[grp];
    const double *com = L.com + 3 * (grp / L.P);
    const double ga = 3.14159265358979323846 * (3.0 - sqrt(5.0));
    float *th = theta + (size_t)pk * 8;
    th[7] = 0.f;
    double u[3];
    const int n_above = mode == 1 ? min(6, K) : 0, nq = K - n_above;
    if (j >= nq) {
        // above the object, approach axis -z (pi about x), yawed by (j - nq) * 60 degrees
        double sh, ch;
        sincos((j - nq) * (3.14159265358979323846 / 6.0), &sh, &ch);
        th[0] = (float)com[0];
        th[1] = (float)com[1];
        th[2] = (float)(com[2] + (double)radius);
        th[3] = 0.f; th[4] = (float)ch; th[5] = (float)sh; th[6] = 0.f;
        return;
    }
    if (mode == 1) {   // quarter sphere facing +x, upper half
        const double z = 1.0 - (j + 0.5) / nq;
        const double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double sa, ca;
        sincos(fmod(j * ga, 3.14159265358979323846) - 0.5 * 3.14159265358979323846, &sa, &ca);
        u[0] = rho * ca; u[1] = rho * sa; u[2] = z;
    } else {
        const double z = 1.0 - (2.0 * j + 1.0) / K;
        const double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double sa, ca;
        sincos(j * ga, &sa, &ca);
        u[0] = rho * ca; u[1] = rho * sa; u[2] = z;
    }
    for (int a = 0; a < 3; ++a) th[a] = (float)(com[a] + (double)radius * u[a]);
    const double w = 1.0 - u[2];
    if (w < 1e-12) {
        th[3] = 0.f; th[4] = 1.f; th[5] = 0.f; th[6] = 0.f;
    } else {
        const double qv[4] = {w, u[1], -u[0], 0.0};
        const double n = sqrt(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2]);
        for (int a = 0; a < 4; ++a) th[3 + a] = (float)(qv[a] / n);
    }
}

cudaError_t launch_fibonacci(const Layout &L, float radius, int mode, float *theta, cudaStream_t st)
{
    fibonacci_kernel<<<(L.T + 255) / 256, 256, 0, st>>>(L, radius, mode, theta);
    return cudaGetLastError();
}

// out[i] = R[idx[i]], i < n (a mini-batch of the object cloud)
__global__ void gather_points_kernel(const float4 *R, const int *idx, int n, float4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = R[idx[i]];
}

cudaError_t launch_gather_points(const float4 *R, const int *idx, int n, float4 *out, cudaStream_t st)
{
    gather_points_kernel<<<(n + 255) / 256, 256, 0, st>>>(R, idx, n, out);
    return cudaGetLastError();
}

__global__ void store_meta_kernel(ObjMeta *dst, const ObjMeta v) { *dst = v; }

cudaError_t launch_store_meta(ObjMeta *dst, const ObjMeta &v, cudaStream_t st)
{
    store_meta_kernel<<<1, 1, 0, st>>>(dst, v);
    return cudaGetLastError();
}

// Particle -> group map and group offsets for P groups of K particles (one object).
__global__ void uniform_groups_kernel(int *part_grp, int *grp_off, int P, int K)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P * K) part_grp[i] = i / K;
    if (i <= P) grp_off[i] = i * K;
}

cudaError_t launch_uniform_groups(int *part_grp, int *grp_off, int P, int K, cudaStream_t st)
{
    const int n = P * K + 1;
    uniform_groups_kernel<<<(n + 255) / 256, 256, 0, st>>>(part_grp, grp_off, P, K);
    return cudaGetLastError();
}

__global__ void set_theta_kernel(const float *theta7, int PK, float *theta8, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= PK) return;
    const float *s = theta7 + (size_t)i * 7;
    float *d = theta8 + (size_t)i * 8;
    bool ok = true;
    for (int a = 0; a < 7; ++a) ok = ok && isfinite(s[a]);
    const double n = sqrt((double)s[3] * s[3] + (double)s[4] * s[4] + (double)s[5] * s[5] + (double)s[6] * s[6]);
    if (!ok || !(n > 0.0)) {
        atomicExch(err, kDevNonFinite);
        return;
    }
    for (int a = 0; a < 3; ++a) d[a] = s[a];
    for (int a = 0; a < 4; ++a) d[3 + a] = (float)((double)s[3 + a] / n);
    d[7] = 0.f;
}

cudaError_t launch_set_theta(const float *theta7, int T, float *theta8, int *err, cudaStream_t st)
{
    set_theta_kernel<<<(T + 255) / 256, 256, 0, st>>>(theta7, T, theta8, err);
    return cudaGetLastError();
}

// Ranking for Algorithm 1's argmin: non-colliding first, ascending cost (NaN
// last), ties to the lower flat index.  Each particle counts the particles that
// precede it, which gives a dense, deterministic order.  The sort key packs the
// collision flag above the cost's order-preserving bit pattern (costs are >= 0).
constexpr int kSelectSmem = 8192;

__device__ __forceinline__ unsigned long long select_key(const double *cost, const int *ncol, int i)
{
    double v = cost[i];
    if (isnan(v) || v < 0.0) v = __longlong_as_double(0x7ff0000000000000LL);
    return ((unsigned long long)(ncol[i] > 0) << 63) | (unsigned long long)__double_as_longlong(v);
}

// One CTA per object: ranks the object's particles; order[pfirst + r] is the
// global index of the particle of rank r.
__global__ void select_kernel(const Layout L, const double *cost, const int *ncol, int *order)
{
    __shared__ unsigned long long keys[kSelectSmem];
    const ObjMeta &om = L.obj[blockIdx.x];
    const int total = om.np;
    const double *c = cost + om.pfirst;
    const int *nc = ncol + om.pfirst;
    const bool staged = total <= kSelectSmem;
    if (staged)
        for (int i = threadIdx.x; i < total; i += blockDim.x) keys[i] = select_key(c, nc, i);
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const unsigned long long ki = staged ? keys[i] : select_key(c, nc, i);
        int rank = 0;
        for (int k = 0; k < total; ++k) {
            const unsigned long long kk = staged ? keys[k] : select_key(c, nc, k);
            rank += kk < ki || (kk == ki && k < i);
        }
        order[om.pfirst + rank] = om.pfirst + i;
    }
}

cudaError_t launch_select(const Layout &L, const double *cost, const int *ncol, int *order, cudaStream_t st)
{
    select_kernel<<<L.nobj, 1024, 0, st>>>(L, cost, ncol, order);
    return cudaGetLastError();
}

}  // namespace asicp
