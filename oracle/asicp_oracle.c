/*
 * FP64 oracle for one AS-ICP iteration ("Grasping by Parallel Shape Matching",
 * arXiv 2412.08346).  TEST INFRASTRUCTURE ONLY: the CUDA path never includes,
 * links or calls it; only tests/, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code with the GPU path.
 *
 * The method is an iteration, so this file performs the paper's steps in the
 * paper's order, with brute-force loops and no blocking or reordering:
 * transform (Alg. 1), nearest neighbour (Eq. 1), match cost and gradient
 * (Eqs. 13-17), SDF collision test (Eq. 12, Section IV-C), collision cost and
 * gradient (Eq. 18 with Eqs. 4-5), annealing (Eq. 11), Stein direction
 * (Eqs. 6, 8-10), SVGD / SGD-ICP updates (Eqs. 7, 3) and the final argmin
 * (Alg. 1).  Where the paper is silent or ambiguous the reading taken is named
 * at the point of use.
 *
 * The paper prints no worked example, intermediate value or trajectory, so the
 * pins in tests/test_oracle_pins.py are closed forms, invariants, library
 * routines and brute force on tiny inputs; the final poses of a whole run are
 * pinned only through such properties (rigid-motion equivariance of whole
 * iterations, recovery of a known rigid transform by SGD-ICP, one SVGD step with
 * K = 1 equal to one SGD step), not against values from the paper.
 */
#include "asicp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Rotation of a quaternion q = (w, x, y, z), homogeneous form
 * R = (w^2 - |v|^2) I + 2 v v^T + 2 w [v]_x  (Section III-A: theta^{4:7} -> R). */
void orc_rotation(const double q[4], double Rm[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double a = w * w - (x * x + y * y + z * z);
    Rm[0] = a + 2 * x * x;     Rm[1] = 2 * x * y - 2 * w * z; Rm[2] = 2 * x * z + 2 * w * y;
    Rm[3] = 2 * x * y + 2 * w * z; Rm[4] = a + 2 * y * y;     Rm[5] = 2 * y * z - 2 * w * x;
    Rm[6] = 2 * x * z - 2 * w * y; Rm[7] = 2 * y * z + 2 * w * x; Rm[8] = a + 2 * z * z;
}

/* d(R(q) s)/dq of the homogeneous form, J is 3x4 row-major with columns
 * (d/dw, d/dx, d/dy, d/dz) (the dR/dq of Eqs. 5 and 17):
 *   d/dw   = 2 w s + 2 v x s
 *   d/dv_k = -2 v_k s + 2 s_k v + 2 (v.s) e_k + 2 w (e_k x s)                */
void orc_rot_jacobian(const double q[4], const double s[3], double J[12])
{
    double w = q[0], v[3] = {q[1], q[2], q[3]};
    double vs = v[0] * s[0] + v[1] * s[1] + v[2] * s[2];
    double vxs[3] = {v[1] * s[2] - v[2] * s[1], v[2] * s[0] - v[0] * s[2], v[0] * s[1] - v[1] * s[0]};
    for (int a = 0; a < 3; ++a)
        J[a * 4 + 0] = 2 * w * s[a] + 2 * vxs[a];
    for (int k = 0; k < 3; ++k) {
        double ek[3] = {0, 0, 0};
        ek[k] = 1.0;
        double exs[3] = {ek[1] * s[2] - ek[2] * s[1], ek[2] * s[0] - ek[0] * s[2], ek[0] * s[1] - ek[1] * s[0]};
        for (int a = 0; a < 3; ++a)
            J[a * 4 + 1 + k] = -2 * v[k] * s[a] + 2 * s[k] * v[a] + 2 * vs * ek[a] + 2 * w * exs[a];
    }
}

static void transform(const double Rm[9], const double t[3], const double s[3], double out[3])
{
    for (int a = 0; a < 3; ++a)
        out[a] = Rm[a * 3 + 0] * s[0] + Rm[a * 3 + 1] * s[1] + Rm[a * 3 + 2] * s[2] + t[a];
}

/* Eq. 1: for every query the reference with the smallest squared distance;
 * ties go to the lowest reference index (reading: the paper gives no rule). */
void orc_nn(const double *Q, int nq, const double *ref, int m, int *idx, double *d2)
{
    for (int i = 0; i < nq; ++i) {
        double best = INFINITY;
        int bi = -1;
        for (int r = 0; r < m; ++r) {
            double dx = Q[i * 3 + 0] - ref[r * 3 + 0];
            double dy = Q[i * 3 + 1] - ref[r * 3 + 1];
            double dz = Q[i * 3 + 2] - ref[r * 3 + 2];
            double d = dx * dx + dy * dy + dz * dz;
            if (d < best) { best = d; bi = r; }
        }
        if (idx) idx[i] = bi;
        if (d2) d2[i] = best;
    }
}

void orc_centroid(const double *X, int n, double c[3])
{
    c[0] = c[1] = c[2] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) c[a] += X[i * 3 + a];
    for (int a = 0; a < 3; ++a) c[a] /= (double)n;
}

/* The problem's CoM: given, or the centroid of its object cloud R. */
static void problem_com(const orc_problem *pb, double com[3])
{
    if (pb->com)
        for (int a = 0; a < 3; ++a) com[a] = pb->com[a];
    else
        orc_centroid(pb->R, pb->M, com);
}

/* Trilinear interpolation of a node-centred grid (x fastest).  A point outside
 * the grid's node box is reported with *inside = 0 (reading: the grid covers
 * the gripper, so such a point cannot be inside it). */
double orc_trilinear(const double *grid, const int dims[3], const double origin[3],
                     double voxel, const double x[3], int *inside)
{
    double u[3], f[3];
    int i0[3];
    *inside = 1;
    for (int a = 0; a < 3; ++a) {
        u[a] = (x[a] - origin[a]) / voxel;
        if (!(u[a] >= 0.0 && u[a] <= (double)(dims[a] - 1))) { *inside = 0; return -INFINITY; }
        int c = (int)floor(u[a]);
        if (c > dims[a] - 2) c = dims[a] - 2;
        if (c < 0) c = 0;
        i0[a] = c;
        f[a] = u[a] - c;
    }
    double v = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double wgt = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                long long id = (long long)(i0[0] + dx) +
                               (long long)dims[0] * ((long long)(i0[1] + dy) + (long long)dims[1] * (i0[2] + dz));
                v += wgt * grid[id];
            }
    return v;
}

static void project_tangent(const double q[4], double g[4])
{
    double d = g[0] * q[0] + g[1] * q[1] + g[2] * q[2] + g[3] * q[3];
    for (int a = 0; a < 4; ++a) g[a] -= d * q[a];
}

/* Match cost and gradient of one particle (Eqs. 13-17) for given pairs
 * (gripper point i <-> object point nn_idx[i]).
 * Readings: the pairs are one per gripper point (N of them) matched against the
 * whole object cloud; the TCP-CoM term sits inside the 1/N with weight w_com as
 * Eqs. 16-17 print it, and the cost is the matching function of that gradient,
 * L = (1/N)(sum |s'_i - r_i|^2 + w_com |R TCP + t - CoM|^2), so the gradient is
 * half of dL/dtheta.  The quaternion block is projected onto the tangent space
 * of the unit sphere at q. */
void orc_match_terms(const orc_problem *pb, int p, const double theta[7], const int *nn_idx,
                     double *cost, double g[7])
{
    const int N = pb->N;
    const double *S = pb->S + (size_t)p * N * 3;
    const double *t = theta, *q = theta + 3;
    double Rm[9], tcp[3], com[3];
    orc_rotation(q, Rm);
    orc_centroid(S, N, tcp);            /* TCP: centre of the contact cloud */
    problem_com(pb, com);               /* CoM: centroid of the object cloud */
    double se = 0.0, ge[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    for (int i = 0; i < N; ++i) {
        double sp[3], J[12];
        const int r = nn_idx[i];
        transform(Rm, t, S + i * 3, sp);
        double e[3] = {sp[0] - pb->R[r * 3 + 0], sp[1] - pb->R[r * 3 + 1], sp[2] - pb->R[r * 3 + 2]};
        se += e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        for (int a = 0; a < 3; ++a) ge[a] += e[a];
        orc_rot_jacobian(q, S + i * 3, J);
        for (int k = 0; k < 4; ++k)
            gq[k] += J[0 * 4 + k] * e[0] + J[1 * 4 + k] * e[1] + J[2 * 4 + k] * e[2];
    }
    {
        double c[3], J[12];
        transform(Rm, t, tcp, c);
        double e[3] = {c[0] - com[0], c[1] - com[1], c[2] - com[2]};
        se += pb->w_com * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        for (int a = 0; a < 3; ++a) ge[a] += pb->w_com * e[a];
        orc_rot_jacobian(q, tcp, J);
        for (int k = 0; k < 4; ++k)
            gq[k] += pb->w_com * (J[0 * 4 + k] * e[0] + J[1 * 4 + k] * e[1] + J[2 * 4 + k] * e[2]);
    }
    *cost = se / N;
    for (int a = 0; a < 3; ++a) g[a] = ge[a] / N;
    for (int k = 0; k < 4; ++k) gq[k] /= N;
    project_tangent(q, gq);
    for (int k = 0; k < 4; ++k) g[3 + k] = gq[k];
}

/* Algorithm 1 for one particle: transform the contact cloud, pair every point
 * with its nearest object point (Eq. 1), then the cost and gradient above. */
void orc_match_cost_grad(const orc_problem *pb, int p, const double theta[7],
                         double *cost, double g[7], int *nn_idx)
{
    const int N = pb->N;
    const double *S = pb->S + (size_t)p * N * 3;
    double Rm[9];
    orc_rotation(theta + 3, Rm);
    int *idx = nn_idx ? nn_idx : (int *)malloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        double sp[3], d2;
        transform(Rm, theta, S + i * 3, sp);
        orc_nn(sp, 1, pb->R, pb->M, idx + i, &d2);
    }
    orc_match_terms(pb, p, theta, idx, cost, g);
    if (!nn_idx) free(idx);
}

/* Collision test (Eq. 12, Section IV-C): each point c of the collision cloud is
 * mapped into the particle's gripper frame, c' = R^T (c - t), and looked up in
 * the preshape's SDF; it collides when the interpolated value is > 0 (positive
 * inside the gripper).  Returns N_col and the colliding indices ascending. */
int orc_collision_points(const orc_problem *pb, int p, const double theta[7],
                         int *list, double *sdf_val)
{
    const double *t = theta, *q = theta + 3;
    double Rm[9];
    orc_rotation(q, Rm);
    const double *grid = pb->sdf + pb->sdf_off[p];
    const int *dims = pb->sdf_dims + 3 * p;
    const double *org = pb->sdf_origin + 3 * p;
    int n = 0;
    for (int c = 0; c < pb->Mc; ++c) {
        double d[3] = {pb->C[c * 3 + 0] - t[0], pb->C[c * 3 + 1] - t[1], pb->C[c * 3 + 2] - t[2]};
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = Rm[0 * 3 + a] * d[0] + Rm[1 * 3 + a] * d[1] + Rm[2 * 3 + a] * d[2];
        int inside;
        double v = orc_trilinear(grid, dims, org, pb->sdf_voxel[p], x, &inside);
        if (sdf_val) sdf_val[c] = v;
        if (inside && v > 0.0) {
            if (list) list[n] = c;
            ++n;
        }
    }
    return n;
}

/* Collision cost and gradient (Eq. 18) for given pairs: colliding point
 * list[l] <-> gripper point nn[l].  L_col = (1/N_col) sum |c - s'|^2, and the
 * gradient follows Eqs. 4-5 with the residual e = s' - c taken with respect to
 * the gripper point s' = R s + t, normalised by N_col and projected like the
 * match gradient. */
void orc_collision_terms(const orc_problem *pb, int p, const double theta[7], const int *list,
                         const int *nn, int ncol, double *cost, double g[7])
{
    const int N = pb->N;
    const double *S = pb->S + (size_t)p * N * 3;
    const double *t = theta, *q = theta + 3;
    double Rm[9];
    orc_rotation(q, Rm);
    double se = 0.0, ge[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    for (int l = 0; l < ncol; ++l) {
        const double *c = pb->C + (size_t)list[l] * 3;
        const int i = nn[l];
        double sp[3], J[12];
        transform(Rm, t, S + i * 3, sp);
        double e[3] = {sp[0] - c[0], sp[1] - c[1], sp[2] - c[2]};
        se += e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        for (int a = 0; a < 3; ++a) ge[a] += e[a];
        orc_rot_jacobian(q, S + i * 3, J);
        for (int k = 0; k < 4; ++k)
            gq[k] += J[0 * 4 + k] * e[0] + J[1 * 4 + k] * e[1] + J[2 * 4 + k] * e[2];
    }
    *cost = se / ncol;
    for (int a = 0; a < 3; ++a) g[a] = ge[a] / ncol;
    for (int k = 0; k < 4; ++k) gq[k] /= ncol;
    project_tangent(q, gq);
    for (int k = 0; k < 4; ++k) g[3 + k] = gq[k];
}

/* Section IV-C: every colliding point is paired with its nearest transformed
 * contact point s' (ties to the lowest gripper index), then the terms above. */
void orc_collision_cost_grad(const orc_problem *pb, int p, const double theta[7],
                             const int *list, int ncol, double *cost, double g[7], int *col_nn)
{
    const int N = pb->N;
    const double *S = pb->S + (size_t)p * N * 3;
    double Rm[9];
    orc_rotation(theta + 3, Rm);
    double *Sp = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    for (int i = 0; i < N; ++i) transform(Rm, theta, S + i * 3, Sp + i * 3);
    int *nn = col_nn ? col_nn : (int *)malloc(sizeof(int) * (size_t)(ncol > 0 ? ncol : 1));
    for (int l = 0; l < ncol; ++l) {
        double d2;
        orc_nn(pb->C + (size_t)list[l] * 3, 1, Sp, N, nn + l, &d2);
    }
    free(Sp);
    orc_collision_terms(pb, p, theta, list, nn, ncol, cost, g);
    if (!col_nn) free(nn);
}

/* Eq. 11: gamma(t) = (mod(t, T/C) / (T/C))^p with T = k_max (cyclic), or the
 * linear ramp g0 -> g1 over the k_max iterations. */
double orc_gamma(const orc_schedule *sc, int k)
{
    if (sc->schedule == 1) {
        if (sc->k_max <= 1) return sc->g1;
        return sc->g0 + (sc->g1 - sc->g0) * (double)k / (double)(sc->k_max - 1);
    }
    double period = (double)sc->k_max / sc->C_cycles;
    return pow(fmod((double)k, period) / period, sc->p_exp);
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Bandwidth h of the RBF kernel (Eq. 9).  The paper gives no value; reading:
 * the SVGD median heuristic, h = med / ln K with med the lower median of the
 * K(K-1)/2 squared translation distances, h = 1 for K = 1, h >= 1e-12. */
double orc_bandwidth(const double *theta, int K, const orc_schedule *sc)
{
    if (sc->bandwidth_mode == 1) return sc->h_fixed;
    if (K < 2) return 1.0;
    size_t L = (size_t)K * (K - 1) / 2, n = 0;
    double *d = (double *)malloc(sizeof(double) * L);
    for (int i = 0; i < K; ++i)
        for (int j = i + 1; j < K; ++j) {
            double dx = theta[i * 7 + 0] - theta[j * 7 + 0];
            double dy = theta[i * 7 + 1] - theta[j * 7 + 1];
            double dz = theta[i * 7 + 2] - theta[j * 7 + 2];
            d[n++] = dx * dx + dy * dy + dz * dz;
        }
    qsort(d, L, sizeof(double), cmp_double);
    double med = d[(L - 1) / 2];
    free(d);
    double h = med / log((double)K);
    return h > 1e-12 ? h : 1e-12;
}

/* Stein direction of Eq. 8 for the K particles of one preshape, read with the
 * expectation of Eq. 6 (a mean over j), the prior term off, and the kernels of
 * Eqs. 9-10 applied per block:
 *   phi_t(i) = (1/K) sum_j [ k_t(j,i) (-gamma N g_t(j)) + (2/h)(t_i - t_j) k_t(j,i) ]
 *   phi_q(i) = (1/K) sum_j [ (q_j.q_i) (-gamma N g_q(j)) + sign(q_j.q_i) q_i ]
 * k_t = exp(-|t_i - t_j|^2 / h); k_r = |q_j.q_i|, whose gradient in q_j is
 * sign(q_j.q_i) q_i.  The drive is multiplied by that same sign (k_r times the
 * sign is q_j.q_i) so that q_j and -q_j, one rotation, push q_i the same way.
 * phi_q is projected onto the tangent space at q_i, which removes the radial
 * rotational repulsion entirely. */
/* Eq. 8 with the priors of Section IV-A (reading R10b): the drive of particle j is
 * gamma (-N g_j + grad log p(theta_j)), the annealing factor scaling both as Eq. 8
 * groups them, with a Gaussian prior on t, grad = -(t - CoM) / sigma^2, and a von
 * Mises prior on the rotation, log p = kappa |mu.q| (q and -q alike), grad = kappa
 * sign(mu.q) mu for the unit mean mu.  prior = {sigma, kappa, mu (4), CoM (3)} or
 * NULL; sigma <= 0 or kappa <= 0 switches a prior off. */
void orc_stein_direction_prior(const double *theta, const double *grad, int K, int N,
                               double gamma, double h, const double *prior, double *phi)
{
    const double sig = prior ? prior[0] : 0.0, kap = prior ? prior[1] : 0.0;
    double mu[4] = {1.0, 0.0, 0.0, 0.0};
    if (prior && kap > 0.0) {
        double n = sqrt(prior[2] * prior[2] + prior[3] * prior[3] + prior[4] * prior[4] + prior[5] * prior[5]);
        for (int a = 0; a < 4; ++a) mu[a] = prior[2 + a] / n;
    }
    for (int i = 0; i < K; ++i) {
        const double *ti = theta + i * 7, *qi = theta + i * 7 + 3;
        double ft[3] = {0, 0, 0}, fq[4] = {0, 0, 0, 0};
        for (int j = 0; j < K; ++j) {
            const double *tj = theta + j * 7, *qj = theta + j * 7 + 3;
            const double *gj = grad + j * 7;
            double drive[7];
            for (int a = 0; a < 7; ++a) drive[a] = -N * gj[a];
            if (sig > 0.0)
                for (int a = 0; a < 3; ++a) drive[a] -= (tj[a] - prior[6 + a]) / (sig * sig);
            if (kap > 0.0) {
                double m = mu[0] * qj[0] + mu[1] * qj[1] + mu[2] * qj[2] + mu[3] * qj[3];
                double sm = m < 0.0 ? -1.0 : 1.0;
                for (int a = 0; a < 4; ++a) drive[3 + a] += kap * sm * mu[a];
            }
            double dt[3] = {ti[0] - tj[0], ti[1] - tj[1], ti[2] - tj[2]};
            double kt = exp(-(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]) / h);
            for (int a = 0; a < 3; ++a)
                ft[a] += kt * (gamma * drive[a]) + (2.0 / h) * dt[a] * kt;
            double c = qj[0] * qi[0] + qj[1] * qi[1] + qj[2] * qi[2] + qj[3] * qi[3];
            double sg = c < 0.0 ? -1.0 : 1.0;
            for (int a = 0; a < 4; ++a)
                fq[a] += c * (gamma * drive[3 + a]) + sg * qi[a];
        }
        for (int a = 0; a < 3; ++a) ft[a] /= K;
        for (int a = 0; a < 4; ++a) fq[a] /= K;
        project_tangent(qi, fq);
        for (int a = 0; a < 3; ++a) phi[i * 7 + a] = ft[a];
        for (int a = 0; a < 4; ++a) phi[i * 7 + 3 + a] = fq[a];
    }
}

void orc_stein_direction(const double *theta, const double *grad, int K, int N,
                         double gamma, double h, double *phi)
{
    orc_stein_direction_prior(theta, grad, K, N, gamma, h, NULL, phi);
}

static void normalize_q(double *q)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) q[a] /= n;
}

/* Fibonacci sphere initialisation (Section V): K directions u_j with
 * z = 1 - (2j+1)/K and golden-angle azimuth j*pi*(3 - sqrt 5); t_j = CoM +
 * radius * u_j; q_j the smallest rotation taking the approach axis +z to -u_j
 * (half-vector form), pi about x when -u_j = -z.  Reading: the full sphere is
 * the default; the paper's quarter sphere and six extra poses are orc_quarter_init. */
void orc_fibonacci_init(int K, const double com[3], double radius, double *theta)
{
    const double ga = M_PI * (3.0 - sqrt(5.0));
    for (int j = 0; j < K; ++j) {
        double z = 1.0 - (2.0 * j + 1.0) / K;
        double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double u[3] = {rho * cos(j * ga), rho * sin(j * ga), z};
        double *th = theta + j * 7;
        for (int a = 0; a < 3; ++a) th[a] = com[a] + radius * u[a];
        double b[3] = {-u[0], -u[1], -u[2]};
        double w = 1.0 + b[2];
        if (w < 1e-12) {
            th[3] = 0.0; th[4] = 1.0; th[5] = 0.0; th[6] = 0.0;
        } else {
            th[3] = w; th[4] = -b[1]; th[5] = b[0]; th[6] = 0.0;
            normalize_q(th + 3);
        }
    }
}

/* Variant of the initialisation used in the paper's experiments (Section VI-A,
 * Fig. 3 (b)): Fibonacci points on the quarter of the sphere facing the robot,
 * plus six initialisations directly above the object.  Readings: the quarter is
 * z >= 0 and x >= 0 relative to the CoM (robot along +x); the lattice is the
 * spiral z_j = 1 - (j + 1/2)/n, azimuth (j * golden angle mod pi) - pi/2, which is
 * uniform in area on that quarter; the last min(6, K) particles sit at
 * CoM + radius e_z, approach axis -e_z, yawed by 0, 60, ..., 300 degrees. */
void orc_quarter_init(int K, const double com[3], double radius, double *theta)
{
    const double ga = M_PI * (3.0 - sqrt(5.0));
    const int n_above = K < 6 ? K : 6, nq = K - n_above;
    for (int j = 0; j < K; ++j) {
        double *th = theta + j * 7;
        if (j < nq) {
            double z = 1.0 - (j + 0.5) / nq;
            double rho = sqrt(fmax(0.0, 1.0 - z * z));
            double phi = fmod(j * ga, M_PI) - 0.5 * M_PI;
            double u[3] = {rho * cos(phi), rho * sin(phi), z};
            for (int a = 0; a < 3; ++a) th[a] = com[a] + radius * u[a];
            th[3] = 1.0 - u[2]; th[4] = u[1]; th[5] = -u[0]; th[6] = 0.0;   /* +z -> -u */
            normalize_q(th + 3);
        } else {
            double half = (j - nq) * M_PI / 6.0;     /* half of the yaw angle */
            th[0] = com[0]; th[1] = com[1]; th[2] = com[2] + radius;
            th[3] = 0.0; th[4] = cos(half); th[5] = sin(half); th[6] = 0.0;  /* yaw about z after pi about x */
        }
    }
}

/* Distances to the nearest and second-nearest of m reference points (plain
 * definition of Eq. 1's minimum, extended to the runner-up). */
static void nearest_two(const double q[3], const double *ref, int m, double *d1, double *d2)
{
    double b1 = INFINITY, b2 = INFINITY;
    for (int r = 0; r < m; ++r) {
        double dx = q[0] - ref[r * 3 + 0], dy = q[1] - ref[r * 3 + 1], dz = q[2] - ref[r * 3 + 2];
        double d = dx * dx + dy * dy + dz * dz;
        if (d < b1) { b2 = b1; b1 = d; }
        else if (d < b2) b2 = d;
    }
    *d1 = sqrt(b1);
    *d2 = sqrt(b2);
}

/* How far the discrete decisions of one step at pose theta are from changing:
 * the smallest of (a) over gripper points, the distance to the second-nearest
 * object point minus the distance to the nearest (Eq. 1), (b) over collision
 * points inside the grid, |SDF value| (the collision test of Eq. 12 flips at 0),
 * (c) over colliding points, the gap between their nearest and second-nearest
 * gripper points (Eq. 18).  All in metres: moving the gripper points, or a
 * point against the SDF (|grad SDF| <= 1 for a distance field), by less than
 * half of it changes none of them.  Used by the tests to tell apart the
 * particles whose trajectory may fork under rounding.  Reported, not used by
 * the method. */
double orc_decision_margin(const orc_problem *pb, int p, const double theta[7])
{
    const int N = pb->N;
    const double *S = pb->S + (size_t)p * N * 3;
    double Rm[9];
    orc_rotation(theta + 3, Rm);
    double *Sp = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) transform(Rm, theta, S + i * 3, Sp + i * 3);
    double margin = INFINITY;
    for (int i = 0; i < N; ++i) {
        double d1, d2;
        nearest_two(Sp + i * 3, pb->R, pb->M, &d1, &d2);
        if (d2 - d1 < margin) margin = d2 - d1;
    }
    const double *grid = pb->sdf + pb->sdf_off[p];
    const int *dims = pb->sdf_dims + 3 * p;
    const double *org = pb->sdf_origin + 3 * p;
    for (int c = 0; c < pb->Mc; ++c) {
        const double *cp = pb->C + (size_t)c * 3;
        double d[3] = {cp[0] - theta[0], cp[1] - theta[1], cp[2] - theta[2]};
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = Rm[0 * 3 + a] * d[0] + Rm[1 * 3 + a] * d[1] + Rm[2 * 3 + a] * d[2];
        int inside;
        double v = orc_trilinear(grid, dims, org, pb->sdf_voxel[p], x, &inside);
        if (!inside) continue;
        if (fabs(v) < margin) margin = fabs(v);
        if (v > 0.0) {
            double d1, d2;
            nearest_two(cp, Sp, N, &d1, &d2);
            if (d2 - d1 < margin) margin = d2 - d1;
        }
    }
    free(Sp);
    return margin;
}

static void particle_cost_grad(const orc_problem *pb, const orc_state *st, int p, int j,
                               double *cost, double g[7], int *ncol)
{
    const int K = pb->K;
    size_t pj = (size_t)p * K + j;
    const double *th = st->theta + pj * 7;
    int *list = st->col_list ? st->col_list + pj * pb->Mc : (int *)malloc(sizeof(int) * (size_t)(pb->Mc > 0 ? pb->Mc : 1));
    double *sv = st->sdf_val ? st->sdf_val + pj * pb->Mc : NULL;
    orc_match_cost_grad(pb, p, th, cost, g, st->nn_idx ? st->nn_idx + pj * pb->N : NULL);
    int n = orc_collision_points(pb, p, th, list, sv);
    if (n > 0)   /* Alg. 1: the collision gradient replaces the match gradient */
        orc_collision_cost_grad(pb, p, th, list, n, cost, g, st->col_nn ? st->col_nn + pj * pb->Mc : NULL);
    *ncol = n;
    if (!st->col_list) free(list);
    if (st->margin) st->margin[pj] = orc_decision_margin(pb, p, th);
}

/* One iteration k of Algorithm 1 for every preshape and particle. */
void orc_step(const orc_problem *pb, const orc_schedule *sc, orc_state *st, int k, int nthreads)
{
    const int P = pb->P, K = pb->K, total = P * K;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int pj = 0; pj < total; ++pj)
        particle_cost_grad(pb, st, pj / K, pj % K, st->cost + pj, st->grad + (size_t)pj * 7, st->ncol + pj);

    const int svgd = k < sc->k_stein;
    /* Convergence (Section IV-D, Table I): in the SGD phase a particle whose
     * relative cost change falls below conv_tol stops updating; a collision
     * clears the flag. */
    for (int pj = 0; pj < total; ++pj) {
        if (!svgd && sc->conv_tol >= 0.0) {
            if (st->ncol[pj] > 0) st->frozen[pj] = 0;
            else if (st->prev_cost[pj] >= 0.0 &&
                     fabs(st->cost[pj] - st->prev_cost[pj]) <= sc->conv_tol * st->prev_cost[pj])
                st->frozen[pj] = 1;
        }
        st->prev_cost[pj] = st->cost[pj];
    }
    memset(st->phi, 0, sizeof(double) * 7 * (size_t)total);
    for (int p = 0; p < P; ++p) {
        double *th = st->theta + (size_t)p * K * 7;
        const double *gr = st->grad + (size_t)p * K * 7;
        if (svgd) {
            double gamma = orc_gamma(sc, k);
            double h = orc_bandwidth(th, K, sc);
            st->h[p] = h;
            double *phi = st->phi + (size_t)p * K * 7;
            double prior[9] = {sc->prior_t_sigma, sc->prior_q_kappa, sc->prior_q_mean[0], sc->prior_q_mean[1],
                               sc->prior_q_mean[2], sc->prior_q_mean[3], 0.0, 0.0, 0.0};
            problem_com(pb, prior + 6);
            orc_stein_direction_prior(th, gr, K, pb->N, gamma, h, prior, phi);
            for (int j = 0; j < K; ++j) {           /* Eq. 7 */
                for (int a = 0; a < 7; ++a) th[j * 7 + a] += sc->eta_svgd * phi[j * 7 + a];
                normalize_q(th + j * 7 + 3);
            }
        } else {
            st->h[p] = 0.0;
            for (int j = 0; j < K; ++j) {           /* Eq. 3 with A = I */
                if (st->frozen[p * K + j]) continue;
                for (int a = 0; a < 7; ++a) th[j * 7 + a] -= sc->eta_sgd * gr[j * 7 + a];
                normalize_q(th + j * 7 + 3);
            }
        }
    }
}

/* Cost and collision count at the current poses, without an update (the
 * final evaluation before the argmin of Alg. 1). */
void orc_evaluate(const orc_problem *pb, orc_state *st, int nthreads)
{
    const int total = pb->P * pb->K;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int pj = 0; pj < total; ++pj)
        particle_cost_grad(pb, st, pj / pb->K, pj % pb->K, st->cost + pj, st->grad + (size_t)pj * 7, st->ncol + pj);
}

/* Alg. 1's argmin, extended to a ranking: non-colliding particles first, then
 * ascending cost, ties to the lower flat index p*K + j. */
void orc_select(const double *cost, const int *ncol, int total, int topk, int *order)
{
    int n = 0;
    for (int r = 0; r < topk && r < total; ++r) {
        int best = -1;
        for (int i = 0; i < total; ++i) {
            int taken = 0;
            for (int s = 0; s < n; ++s) if (order[s] == i) { taken = 1; break; }
            if (taken) continue;
            if (best < 0) { best = i; continue; }
            int ci = ncol[i] > 0, cb = ncol[best] > 0;
            if (ci < cb || (ci == cb && cost[i] < cost[best])) best = i;
        }
        order[n++] = best;
    }
}
