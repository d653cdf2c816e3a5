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

#define ORC_MAXB 32
#define ORC_MAXV 38
#define ORC_MAXQ 39
#define ORC_MAXCAND 4096
#define ORC_CAPMAX 128
#define ORC_NPHASE 9

enum { ORC_PH_CPG = 0, ORC_PH_FK, ORC_PH_RNEA, ORC_PH_CRBA, ORC_PH_CHOL,
       ORC_PH_CONTACT, ORC_PH_JAC, ORC_PH_PGS, ORC_PH_INTEG };

enum { ORC_ST_NONFINITE = 1, ORC_ST_OVERFLOW = 2, ORC_ST_CHOL = 4 };

enum { ORC_GEOM_BOX = 0, ORC_GEOM_SPHERE = 1 };

typedef struct {
    int32_t nb;                 /* bodies, 1..32; body 0 is the root        */
    int32_t root_fixed;         /* 1: root pinned at (root_R, root_p)       */
    int32_t parent[ORC_MAXB];   /* parent[b] < b for b >= 1                 */
    int32_t axis[ORC_MAXB];     /* hinge axis index (0,1,2) in child frame  */
    uint32_t exclude[ORC_MAXB]; /* bit j: body never collides with body j   */
    double R_fix[ORC_MAXB][9];  /* child frame at zero angle, in parent     */
    double p_fix[ORC_MAXB][3];
    double half[ORC_MAXB][3];   /* box half extents (body axes)             */
    double com[ORC_MAXB][3];    /* box centre in body frame                 */
    double mass[ORC_MAXB];
    double w_int[ORC_MAXB];     /* CPG weight of hinge body b               */
    double w_cpl[ORC_MAXB];     /* CPG coupling of hinge b to its parent    */
    double root_R[9];
    double root_p[3];
    int32_t geom[ORC_MAXB];     /* ORC_GEOM_BOX or ORC_GEOM_SPHERE; a sphere
                                   has radius half[b][0], centre com[b]     */
} orc_model;

typedef struct {
    double dt;
    double gravity[3];
    int32_t pgs_iters;
    double soft_tau, soft_zeta, mu;
    int32_t contact_cap;
    double kp, kd, tau_max, theta_max, armature;
    int32_t ground;             /* body/plane contacts on                   */
    int32_t box_box;            /* body/body contacts inside a robot on     */
    int32_t actuate;            /* CPG + PD torques on                      */
    double max_correct_vel;     /* cap of the penetration recovery speed    */
    double min_cfm;             /* floor of a row's softness R [1/kg]       */
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
    double p[ORC_MAXCAND][3];   /* world position                           */
    double nrm[ORC_MAXCAND][3]; /* from body b towards body a               */
    double depth[ORC_MAXCAND];
} orc_contact_list;

#ifdef __cplusplus
extern "C" {
#endif
void orc_default_params(orc_params* p);
int orc_nq(const orc_model* m);
int orc_nv(const orc_model* m);
/* body rotations (row-major), frame origins and box centres in world */
void orc_fk(const orc_model* m, const double* q, double* R, double* p, double* c);
/* joint-space inertia (nv x nv, row-major, armature included) */
void orc_mass_matrix(const orc_model* m, const orc_params* prm, const double* q, double* M);
/* bias force c(q, v) including gravity */
void orc_bias(const orc_model* m, const orc_params* prm, const double* q, const double* v, double* c);
/* dense Cholesky, returns 0 on success, -1 on a non-positive pivot */
int orc_cholesky(int n, const double* M, double* L);
/* contacts of the current configuration, after the cap (returns status bits) */
int orc_contacts(const orc_model* m, const orc_params* prm, const double* q,
                 orc_contact_list* out, double* margin);
/* contact impulses after the soft PGS of one step (for inspection) */
int orc_step_detail(const orc_model* m, const orc_params* prm, double* q, double* v,
                    double* s, uint32_t* status, double* vfree_out, double* lambda_out,
                    int32_t* nc_out);
/* n steps of one variant, in place; stats accumulate (may be NULL) */
int orc_run(const orc_model* m, const orc_params* prm, int nsteps, double* q,
            double* v, double* s, uint32_t* status, orc_stats* st);
/* many variants (model array), nthreads pthreads over variants */
int orc_run_many(const orc_model* m, int nvar, const orc_params* prm, int nsteps,
                 double* q, int q_stride, double* v, int v_stride, double* s, int s_stride,
                 uint32_t* status, orc_stats* st, int nthreads);
int orc_sizeof_model(void);
int orc_sizeof_params(void);
int orc_sizeof_stats(void);
#ifdef __cplusplus
}
#endif
#endif
