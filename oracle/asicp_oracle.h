/*
 * FP64 reference implementation of one AS-ICP iteration ("Grasping by Parallel
 * Shape Matching", arXiv 2412.08346).  TEST INFRASTRUCTURE ONLY: the CUDA path
 * never includes, links or calls this code; only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark use it.
 *
 * Every quantity is float64.  Arrays are row-major, points are xyz triples,
 * poses are theta = (t_x, t_y, t_z, q_w, q_x, q_y, q_z) (Section III-A).
 */
#ifndef ASICP_ORACLE_H
#define ASICP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int P, K, N, M, Mc;
    const double *S;          /* P*N*3  gripper contact clouds (gripper frame)   */
    const double *R;          /* M*3    object cloud (matching, Eq. 1)           */
    const double *C;          /* Mc*3   collision cloud (object [+ table])       */
    const double *sdf;        /* concatenated grids, x fastest, + inside         */
    const long long *sdf_off; /* P offsets (in values) into sdf                  */
    const int *sdf_dims;      /* P*3 (nx, ny, nz)                                */
    const double *sdf_origin; /* P*3 position of node (0,0,0)                    */
    const double *sdf_voxel;  /* P   node spacing                                */
    double w_com;             /* weight of the TCP-CoM term inside 1/N (Eqs. 16-17) */
    const double *com;        /* 3: CoM, or NULL for the centroid of R (a mini-batch
                                 of R keeps the whole object's CoM)                */
} orc_problem;

typedef struct {
    int k_max, k_stein;
    int schedule;             /* 0: cyclic Eq. 11, 1: linear g0 -> g1            */
    double C_cycles, p_exp, g0, g1;
    double eta_sgd, eta_svgd;
    int bandwidth_mode;       /* 0: median heuristic, 1: h_fixed                 */
    double h_fixed;
    double conv_tol;          /* < 0 disables freezing                            */
    double prior_t_sigma;     /* Gaussian prior on t around the CoM (<= 0: off)   */
    double prior_q_kappa;     /* von Mises prior on q (<= 0: off)                 */
    double prior_q_mean[4];   /* its mean rotation (normalised)                   */
} orc_schedule;

typedef struct {
    double *theta;            /* P*K*7  in/out                                    */
    double *cost;             /* P*K    cost at theta before the update           */
    double *grad;             /* P*K*7  gradient used (match or collision)        */
    double *phi;              /* P*K*7  Stein direction (zero in the SGD phase)   */
    int *ncol;                /* P*K    number of colliding points                */
    int *frozen;              /* P*K    convergence flag (in/out)                 */
    double *prev_cost;        /* P*K    in/out, negative = none                   */
    double *h;                /* P      bandwidth used                            */
    int *nn_idx;              /* P*K*N  forward correspondences (nullable)        */
    int *col_list;            /* P*K*Mc colliding point indices, ascending (nullable) */
    int *col_nn;              /* P*K*Mc reverse-NN gripper index per colliding point (nullable) */
    double *sdf_val;          /* P*K*Mc interpolated SDF at every C point (nullable) */
    double *margin;           /* P*K    decision margin of the step (nullable), see
                                 orc_decision_margin                               */
} orc_state;

void orc_rotation(const double q[4], double Rm[9]);
void orc_rot_jacobian(const double q[4], const double s[3], double J[12]);
void orc_nn(const double *Q, int nq, const double *ref, int m, int *idx, double *d2);
double orc_trilinear(const double *grid, const int dims[3], const double origin[3],
                     double voxel, const double x[3], int *inside);
void orc_match_terms(const orc_problem *pb, int p, const double theta[7], const int *nn_idx,
                     double *cost, double g[7]);
void orc_collision_terms(const orc_problem *pb, int p, const double theta[7], const int *list,
                         const int *nn, int ncol, double *cost, double g[7]);
void orc_match_cost_grad(const orc_problem *pb, int p, const double theta[7],
                         double *cost, double g[7], int *nn_idx);
int orc_collision_points(const orc_problem *pb, int p, const double theta[7],
                         int *list, double *sdf_val);
void orc_collision_cost_grad(const orc_problem *pb, int p, const double theta[7],
                             const int *list, int ncol, double *cost, double g[7], int *col_nn);
double orc_gamma(const orc_schedule *sc, int k);
double orc_bandwidth(const double *theta, int K, const orc_schedule *sc);
void orc_stein_direction(const double *theta, const double *grad, int K, int N,
                         double gamma, double h, double *phi);
void orc_stein_direction_prior(const double *theta, const double *grad, int K, int N,
                               double gamma, double h, const double *prior, double *phi);
void orc_fibonacci_init(int K, const double com[3], double radius, double *theta);
void orc_quarter_init(int K, const double com[3], double radius, double *theta);
void orc_centroid(const double *X, int n, double c[3]);
void orc_step(const orc_problem *pb, const orc_schedule *sc, orc_state *st, int k, int nthreads);
void orc_evaluate(const orc_problem *pb, orc_state *st, int nthreads);
void orc_select(const double *cost, const int *ncol, int total, int topk, int *order);
double orc_decision_margin(const orc_problem *pb, int p, const double theta[7]);

#ifdef __cplusplus
}
#endif
#endif
