/*
 * orc.h -- FP64 CPU oracle of the population-stepping hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this code: only tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * The paper (Sec. 2 "Materials", Sec. 4 "Simulation Parameters") benchmarks a
 * simulator stepping many independent *variants* of a scene for a number of
 * steps; it does not print the physics itself.  The step below is therefore
 * built from named textbook methods, one variant at a time, plainly:
 *   - CPG: antisymmetric linear oscillator network, explicit Euler, PD servo;
 *   - forward kinematics down the body tree;
 *   - bias forces c(q,v) by recursive Newton-Euler (Featherstone 2008, ch. 5),
 *     gravity entered as a base acceleration;
 *   - joint-space inertia M(q) by the composite-rigid-body algorithm
 *     (Featherstone 2008, ch. 6), plus a hinge armature;
 *   - dense Cholesky M = L L^T, unconstrained velocity v + dt M^-1 (tau - c);
 *   - contacts: box/plane vertices, box/box by the separating-axis test with
 *     face clipping (Sutherland-Hodgman) or an edge-edge point; sphere/plane,
 *     sphere/box (closest point of the box) and sphere/sphere, one point each;
 *   - soft projected Gauss-Seidel on contact impulses (ODE ERP/CFM soft
 *     constraints, mass-normalised), disk friction cone, fixed sweep count;
 *   - semi-implicit Euler on the configuration (quaternion exponential map).
 * Spatial vectors are expressed in world axes about the point O = the root
 * frame origin at the start of the step; motion vectors are (omega; v_O),
 * force vectors are (n_O; f).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#define ORC_MAXB 64
#define ORC_MAXV 70
#define ORC_MAXQ 71
#define ORC_MAXCAND 4096
#define ORC_CAPMAX 128
#define ORC_NPHASE 9
#define ORC_MAXNEAR 64

enum { ORC_PH_CPG = 0, ORC_PH_FK, ORC_PH_RNEA, ORC_PH_CRBA, ORC_PH_CHOL,
       ORC_PH_CONTACT, ORC_PH_JAC, ORC_PH_PGS, ORC_PH_INTEG };

enum { ORC_ST_NONFINITE = 1, ORC_ST_OVERFLOW = 2, ORC_ST_CHOL = 4 };

enum { ORC_GEOM_BOX = 0, ORC_GEOM_SPHERE = 1 };

/* Scalar type of the oracle's arithmetic: double (the oracle proper).  A
 * second build with ORC_FP32 defined evaluates the same statements in the same
 * order in FP32; it is a yardstick for the rounding error that FP32
 * arithmetic alone brings to this method, and nothing else uses it. */
#ifdef ORC_FP32
#define ORC_REAL float
#else
#define ORC_REAL double
#endif
typedef ORC_REAL real;

typedef struct {
    int32_t nb;                 /* bodies, 1..64; body 0 is the root        */
    int32_t root_fixed;         /* 1: root pinned at (root_R, root_p)       */
    int32_t parent[ORC_MAXB];   /* parent[b] < b for b >= 1                 */
    int32_t axis[ORC_MAXB];     /* hinge axis index (0,1,2) in child frame  */
    uint64_t exclude[ORC_MAXB]; /* bit j: body never collides with body j   */
    real R_fix[ORC_MAXB][9];  /* child frame at zero angle, in parent     */
    real p_fix[ORC_MAXB][3];
    real half[ORC_MAXB][3];   /* box half extents (body axes)             */
    real com[ORC_MAXB][3];    /* box centre in body frame                 */
    real mass[ORC_MAXB];
    real w_int[ORC_MAXB];     /* CPG weight of hinge body b               */
    real w_cpl[ORC_MAXB];     /* CPG coupling of hinge b to its parent    */
    real root_R[9];
    real root_p[3];
    int32_t geom[ORC_MAXB];     /* ORC_GEOM_BOX or ORC_GEOM_SPHERE; a sphere
                                   has radius half[b][0], centre com[b]     */
} orc_model;

typedef struct {
    real dt;
    real gravity[3];
    int32_t pgs_iters;
    real soft_tau, soft_zeta, mu;
    int32_t contact_cap;
    real kp, kd, tau_max, theta_max, armature;
    int32_t ground;             /* body/plane contacts on                   */
    int32_t box_box;            /* body/body contacts inside a robot on     */
    int32_t actuate;            /* CPG + PD torques on                      */
    real max_correct_vel;     /* cap of the penetration recovery speed    */
    real min_cfm;             /* floor of a row's softness R [1/kg]       */
} orc_params;

typedef struct {
    double flops[ORC_NPHASE];   /* algorithmic flops per phase, summed      */
    double contacts;            /* sum over steps of active contacts        */
    double narrow_pairs;        /* sum over steps of box/box narrow phases  */
    double broad_pairs;         /* sum over steps of box/box broad tests    */
    double margin;              /* min distance of any discrete decision to
                                   its threshold (metres or ratio)          */
    int32_t overflow_steps;
    int32_t steps;
} orc_stats;

typedef struct {
    int32_t n;
    int32_t a[ORC_MAXCAND], b[ORC_MAXCAND];
    real p[ORC_MAXCAND][3];   /* world position                           */
    real nrm[ORC_MAXCAND][3]; /* from body b towards body a               */
    real depth[ORC_MAXCAND];
} orc_contact_list;

#ifdef __cplusplus
extern "C" {
#endif
void orc_default_params(orc_params* p);
int orc_nq(const orc_model* m);
int orc_nv(const orc_model* m);
/* body rotations (row-major), frame origins and box centres in world */
void orc_fk(const orc_model* m, const real* q, real* R, real* p, real* c);
/* joint-space inertia (nv x nv, row-major, armature included) */
void orc_mass_matrix(const orc_model* m, const orc_params* prm, const real* q, real* M);
/* bias force c(q, v) including gravity */
void orc_bias(const orc_model* m, const orc_params* prm, const real* q, const real* v, real* c);
/* dense Cholesky, returns 0 on success, -1 on a non-positive pivot */
int orc_cholesky(int n, const real* M, real* L);
/* contacts of the current configuration, after the cap (returns status bits) */
int orc_contacts(const orc_model* m, const orc_params* prm, const real* q,
                 orc_contact_list* out, real* margin);
/* the contact list with near-threshold decisions taken the other way, as in
 * orc_step_flip (returns status bits, or -1 for bad arguments) */
int orc_contacts_flip(const orc_model* m, const orc_params* prm, const real* q, double band,
                      const int32_t* flip, int32_t nflip, orc_contact_list* out, int32_t* near_out,
                      int32_t* nnear_out, double* margin_out);
/* contact impulses after the soft PGS of one step (for inspection) */
int orc_step_detail(const orc_model* m, const orc_params* prm, real* q, real* v,
                    real* s, uint32_t* status, real* vfree_out, real* lambda_out,
                    int32_t* nc_out);
/* One step of one variant, in place, taking some near-threshold decisions
 * the other way (test use: the other valid outcomes of a step whose discrete
 * decisions -- contact activation, separating-axis and incident-face choice,
 * clipping side, cap cut, frozen rows -- lie within `band` of their
 * thresholds, where FP32 and FP64 arithmetic may branch differently).
 * Decisions within band are numbered in the order the step takes them;
 * those listed in flip[0..nflip) are reversed (a near tie takes the
 * runner-up).  near_out (room for ORC_MAXNEAR, may be NULL) receives the
 * numbers met, *nnear_out their count, *margin_out the step's margin.  With
 * nflip = 0 the result is exactly orc_run's for one step.  Returns 0, or -1
 * for bad arguments. */
int orc_step_flip(const orc_model* m, const orc_params* prm, real* q, real* v, real* s, uint32_t* status,
                  double band, const int32_t* flip, int32_t nflip, int32_t* near_out, int32_t* nnear_out,
                  double* margin_out);
/* n steps of one variant, in place; stats accumulate (may be NULL) */
int orc_run(const orc_model* m, const orc_params* prm, int nsteps, real* q,
            real* v, real* s, uint32_t* status, orc_stats* st);
/* many variants (model array), nthreads pthreads over variants */
int orc_run_many(const orc_model* m, int nvar, const orc_params* prm, int nsteps,
                 real* q, int q_stride, real* v, int v_stride, real* s, int s_stride,
                 uint32_t* status, orc_stats* st, int nthreads);
int orc_sizeof_model(void);
int orc_sizeof_params(void);
int orc_sizeof_stats(void);
#ifdef __cplusplus
}
#endif
#endif
