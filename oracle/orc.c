/*
 * orc.c -- FP64 CPU oracle of the population-stepping hot path.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
 * baseline leg are the only callers.  Plain, scalar, one variant at a time,
 * no blocking or fusion beyond the algorithm's own steps.  See orc.h for the
 * list of methods and conventions.
 *
 * Flop counting: every arithmetic statement adds its count of floating point
 * operations (add, sub, mul, div, sqrt, sin, cos, abs, min/max each 1) to the
 * counter of the phase it belongs to.  These counts are the "algorithmic
 * flops" used for roofline accounting.
 *
 * Parity pins: see the header of oracle/oracle.py for which test pins which
 * function.
 */
#include "orc.h"
#include <math.h>
#ifdef ORC_FP32
/* the FP32 yardstick build: single-precision library routines */
#define sqrt sqrtf
#define fabs fabsf
#define sin sinf
#define cos cosf
#endif
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int32_t a[ORC_CAPMAX], b[ORC_CAPMAX];
    real p[ORC_CAPMAX][3], nrm[ORC_CAPMAX][3], depth[ORC_CAPMAX];
} kept_list;

typedef struct {
    real O[3];
    real R[ORC_MAXB][9];
    real r[ORC_MAXB][3];   /* frame origin minus O            */
    real c[ORC_MAXB][3];   /* box centre minus O              */
    real S[ORC_MAXB][6];   /* hinge motion subspace           */
    real vb[ORC_MAXB][6], ab[ORC_MAXB][6], f[ORC_MAXB][6];
    real I[ORC_MAXB][10], Ic[ORC_MAXB][10];
    int nv, nq, dof0, q0h;
    real M[ORC_MAXV * ORC_MAXV], L[ORC_MAXV * ORC_MAXV];
    real cb[ORC_MAXV], tau[ORC_MAXV], vfree[ORC_MAXV], vnew[ORC_MAXV];
    orc_contact_list cand;
    kept_list con;
    real J[3 * ORC_CAPMAX][ORC_MAXV], Wm[3 * ORC_CAPMAX][ORC_MAXV];
    real A[3 * ORC_CAPMAX], Rs[3 * ORC_CAPMAX], tgt[3 * ORC_CAPMAX], lam[3 * ORC_CAPMAX];
    double flops[ORC_NPHASE];
    int phase;
    double margin;
    /* near-threshold decisions (see decide) */
    int dseq;
    double band;
    int nflip, flip[ORC_MAXNEAR];
    int nnear, near[ORC_MAXNEAR];
    int narrow, broad;
} work;

#define ORC_PI 3.14159265358979323846
#define ORC_AMIN 1e-10  /* rows with J M^-1 J^T below this are frozen */
#define ORC_CLIP_ON 1e-6  /* a polygon vertex this close to a clipping plane is on it [m] */
#define FL(w, n) ((w)->flops[(w)->phase] += (double)(n))

static void note_margin(work* w, double m) {
    if (m < 0.0) m = -m;
    if (m < w->margin) w->margin = m;
}

/* A discrete decision of the step whose outcome changes the result
 * discontinuously, at signed distance m from its threshold.  Like
 * note_margin it keeps the step's smallest |m|.  Decisions within w->band of
 * their threshold are numbered in the order the step takes them, so that a
 * caller can ask for another valid outcome of the same step (FP32 and FP64
 * arithmetic may legitimately go either way there): the decisions listed in
 * w->flip are taken the other way.  Returns 1 for a decision to reverse;
 * with band 0 (every ordinary call) it always returns 0. */
static int decide(work* w, double m) {
    note_margin(w, m);
    if (m < 0.0) m = -m;
    if (!(m < w->band)) return 0;
    int id = w->dseq++;
    if (w->nnear < ORC_MAXNEAR) w->near[w->nnear] = id;
    w->nnear++;
    for (int k = 0; k < w->nflip; ++k)
        if (w->flip[k] == id) return 1;
    return 0;
}

/* ---------------------------------------------------------------- helpers */
static real dot3(work* w, const real* a, const real* b) {
    FL(w, 5);
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(work* w, const real* a, const real* b, real* o) {
    real t0 = a[1] * b[2] - a[2] * b[1];
    real t1 = a[2] * b[0] - a[0] * b[2];
    real t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
    FL(w, 9);
}
static void matvec(work* w, const real* R, const real* x, real* o) {
    real t[3];
    for (int i = 0; i < 3; ++i) t[i] = R[3 * i] * x[0] + R[3 * i + 1] * x[1] + R[3 * i + 2] * x[2];
    o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
    FL(w, 15);
}
static void mattvec(work* w, const real* R, const real* x, real* o) {
    real t[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * x[0] + R[3 + i] * x[1] + R[6 + i] * x[2];
    o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
    FL(w, 15);
}
static void matmul(work* w, const real* A, const real* B, real* C) {
    real t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            t[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, t, sizeof t);
    FL(w, 45);
}
static void col(const real* R, int k, real* o) {
    o[0] = R[k]; o[1] = R[3 + k]; o[2] = R[6 + k];
}

/* rotation matrix of a (not re-normalised) quaternion (w, x, y, z) */
static void quat_to_R(work* w, const real* q, real* R) {
    real qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    R[0] = 1 - 2 * (qy * qy + qz * qz); R[1] = 2 * (qx * qy - qw * qz); R[2] = 2 * (qx * qz + qw * qy);
    R[3] = 2 * (qx * qy + qw * qz); R[4] = 1 - 2 * (qx * qx + qz * qz); R[5] = 2 * (qy * qz - qw * qx);
    R[6] = 2 * (qx * qz - qw * qy); R[7] = 2 * (qy * qz + qw * qx); R[8] = 1 - 2 * (qx * qx + qy * qy);
    FL(w, 39);
}

/* rotation by theta about body axis e_k */
static void axis_rot(work* w, int k, real th, real* R) {
    real c = cos(th), s = sin(th);
    FL(w, 2);
    memset(R, 0, 9 * sizeof(real));
    if (k == 0) { R[0] = 1; R[4] = c; R[5] = -s; R[7] = s; R[8] = c; }
    else if (k == 1) { R[0] = c; R[2] = s; R[4] = 1; R[6] = -s; R[8] = c; }
    else { R[0] = c; R[1] = -s; R[3] = s; R[4] = c; R[8] = 1; }
}

/* -------------------------------------------------------- model geometry */
static int model_nv(const orc_model* m) { return (m->root_fixed ? 0 : 6) + m->nb - 1; }
static int model_nq(const orc_model* m) { return (m->root_fixed ? 0 : 7) + m->nb - 1; }
int orc_nv(const orc_model* m) { return model_nv(m); }
int orc_nq(const orc_model* m) { return model_nq(m); }
int orc_sizeof_model(void) { return (int)sizeof(orc_model); }
int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_stats(void) { return (int)sizeof(orc_stats); }

void orc_default_params(orc_params* p) {
    memset(p, 0, sizeof *p);
    p->dt = 0.002;
    p->gravity[2] = -9.81;
    p->pgs_iters = 30;
    p->soft_tau = 0.02;
    p->soft_zeta = 1.0;
    p->mu = 1.0;
    p->contact_cap = 64;
    p->kp = 2.0;
    p->kd = 0.05;
    p->tau_max = 1.0;
    p->theta_max = 1.5707963267948966;
    p->armature = 1e-4;
    p->ground = 1;
    p->box_box = 1;
    p->actuate = 1;
    p->max_correct_vel = 0.1;
    p->min_cfm = 0.1;
}

static void setup(work* w, const orc_model* m) {
    w->nv = model_nv(m);
    w->nq = model_nq(m);
    w->dof0 = m->root_fixed ? 0 : 6;
    w->q0h = m->root_fixed ? 0 : 7;
}

/* ------------------------------------------------------------------- FK
 * R_b = R_parent R_fix,b Rot(axis_b, theta_b);  r_b = r_parent + R_parent p_fix,b.
 * Positions are kept relative to O = root frame origin. */
static void fk(work* w, const orc_model* m, const real* q) {
    w->phase = ORC_PH_FK;
    if (m->root_fixed) {
        memcpy(w->O, m->root_p, sizeof w->O);
        memcpy(w->R[0], m->root_R, 9 * sizeof(real));
    } else {
        memcpy(w->O, q, 3 * sizeof(real));
        quat_to_R(w, q + 3, w->R[0]);
    }
    w->r[0][0] = w->r[0][1] = w->r[0][2] = 0.0;
    for (int b = 1; b < m->nb; ++b) {
        int p = m->parent[b];
        real Rl[9], Ra[9], t[3];
        axis_rot(w, m->axis[b], q[w->q0h + b - 1], Ra);
        matmul(w, m->R_fix[b], Ra, Rl);
        matmul(w, w->R[p], Rl, w->R[b]);
        matvec(w, w->R[p], m->p_fix[b], t);
        for (int k = 0; k < 3; ++k) w->r[b][k] = w->r[p][k] + t[k];
        FL(w, 3);
    }
    for (int b = 0; b < m->nb; ++b) {
        real t[3];
        matvec(w, w->R[b], m->com[b], t);
        for (int k = 0; k < 3; ++k) w->c[b][k] = w->r[b][k] + t[k];
        FL(w, 3);
    }
}

/* hinge motion subspace S_b = (a_b; r_b x a_b), a_b = R_b e_axis */
static void motion_subspaces(work* w, const orc_model* m) {
    for (int b = 1; b < m->nb; ++b) {
        real a[3], ra[3];
        col(w->R[b], m->axis[b], a);
        cross3(w, w->r[b], a, ra);
        w->S[b][0] = a[0]; w->S[b][1] = a[1]; w->S[b][2] = a[2];
        w->S[b][3] = ra[0]; w->S[b][4] = ra[1]; w->S[b][5] = ra[2];
    }
}

/* spatial inertia about O in world axes: (m, h = m c, Irot about O) */
static void body_inertias(work* w, const orc_model* m) {
    for (int b = 0; b < m->nb; ++b) {
        const real* h = m->half[b];
        real mb = m->mass[b];
        /* principal moments about the centre: solid box m (h_j^2 + h_k^2) / 3,
         * solid sphere 2 m r^2 / 5 */
        real Id[3];
        if (m->geom[b] == ORC_GEOM_SPHERE) {
            Id[0] = Id[1] = Id[2] = 0.4 * mb * h[0] * h[0];
            FL(w, 3);
        } else {
            Id[0] = mb * (h[1] * h[1] + h[2] * h[2]) / 3.0;
            Id[1] = mb * (h[0] * h[0] + h[2] * h[2]) / 3.0;
            Id[2] = mb * (h[0] * h[0] + h[1] * h[1]) / 3.0;
            FL(w, 18);
        }
        const real* R = w->R[b];
        real Iw[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Iw[3 * i + j] = R[3 * i] * Id[0] * R[3 * j] + R[3 * i + 1] * Id[1] * R[3 * j + 1] +
                                R[3 * i + 2] * Id[2] * R[3 * j + 2];
        FL(w, 6 * 8);  /* 6 unique entries x (6 mul + 2 add) */
        const real* c = w->c[b];
        real cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        FL(w, 5);
        real* I = w->I[b];
        I[0] = mb;
        I[1] = mb * c[0]; I[2] = mb * c[1]; I[3] = mb * c[2];
        I[4] = Iw[0] + mb * (cc - c[0] * c[0]);
        I[5] = Iw[4] + mb * (cc - c[1] * c[1]);
        I[6] = Iw[8] + mb * (cc - c[2] * c[2]);
        I[7] = Iw[1] - mb * c[0] * c[1];
        I[8] = Iw[2] - mb * c[0] * c[2];
        I[9] = Iw[5] - mb * c[1] * c[2];
        FL(w, 3 + 3 * 4 + 3 * 3);
    }
}

/* f = I * (omega; v) for a spatial inertia stored as (m, h, Irot) */
static void inertia_apply(work* w, const real* I, const real* mv, real* f) {
    const real* om = mv;
    const real* vo = mv + 3;
    real n[3], hv[3], hw[3];
    n[0] = I[4] * om[0] + I[7] * om[1] + I[8] * om[2];
    n[1] = I[7] * om[0] + I[5] * om[1] + I[9] * om[2];
    n[2] = I[8] * om[0] + I[9] * om[1] + I[6] * om[2];
    FL(w, 15);
    cross3(w, I + 1, vo, hv);
    cross3(w, I + 1, om, hw);
    f[0] = n[0] + hv[0]; f[1] = n[1] + hv[1]; f[2] = n[2] + hv[2];
    f[3] = I[0] * vo[0] - hw[0]; f[4] = I[0] * vo[1] - hw[1]; f[5] = I[0] * vo[2] - hw[2];
    FL(w, 3 + 6);
}

/* crm(v) m : motion cross product */
static void crm(work* w, const real* v, const real* mm, real* o) {
    real a[3], b[3], c[3];
    cross3(w, v, mm, a);
    cross3(w, v, mm + 3, b);
    cross3(w, v + 3, mm, c);
    o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
    o[3] = b[0] + c[0]; o[4] = b[1] + c[1]; o[5] = b[2] + c[2];
    FL(w, 3);
}

/* crf(v) f : force cross product */
static void crf(work* w, const real* v, const real* f, real* o) {
    real a[3], b[3], c[3];
    cross3(w, v, f, a);
    cross3(w, v + 3, f + 3, b);
    cross3(w, v, f + 3, c);
    o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2];
    o[3] = c[0]; o[4] = c[1]; o[5] = c[2];
    FL(w, 3);
}

static real sdot(work* w, const real* a, const real* b) {
    FL(w, 11);
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3] + a[4] * b[4] + a[5] * b[5];
}

/* ---------------------------------------------------------------- RNEA
 * c(q, v) = inverse dynamics with zero joint acceleration and the base
 * accelerating at -g (Featherstone 2008, Table 5.1 with a_0 = -g). */
static void rnea(work* w, const orc_model* m, const orc_params* prm, const real* v, real* cb) {
    w->phase = ORC_PH_RNEA;
    const real* g = prm->gravity;
    if (m->root_fixed) {
        memset(w->vb[0], 0, 6 * sizeof(real));
        w->ab[0][0] = w->ab[0][1] = w->ab[0][2] = 0.0;
        w->ab[0][3] = -g[0]; w->ab[0][4] = -g[1]; w->ab[0][5] = -g[2];
    } else {
        /* root twist: angular velocity to world axes, linear velocity of O */
        real om[3], vxw[3];
        matvec(w, w->R[0], v + 3, om);
        w->vb[0][0] = om[0]; w->vb[0][1] = om[1]; w->vb[0][2] = om[2];
        w->vb[0][3] = v[0]; w->vb[0][4] = v[1]; w->vb[0][5] = v[2];
        /* root spatial acceleration at zero qdd: (0; -omega x v_O) */
        cross3(w, v, om, vxw);
        w->ab[0][0] = w->ab[0][1] = w->ab[0][2] = 0.0;
        w->ab[0][3] = vxw[0] - g[0]; w->ab[0][4] = vxw[1] - g[1]; w->ab[0][5] = vxw[2] - g[2];
        FL(w, 3);
    }
    for (int b = 1; b < m->nb; ++b) {
        int p = m->parent[b];
        real qd = v[w->dof0 + b - 1];
        real Sq[6], cr[6];
        for (int k = 0; k < 6; ++k) {
            Sq[k] = w->S[b][k] * qd;
            w->vb[b][k] = w->vb[p][k] + Sq[k];
        }
        FL(w, 12);
        crm(w, w->vb[b], Sq, cr);
        for (int k = 0; k < 6; ++k) w->ab[b][k] = w->ab[p][k] + cr[k];
        FL(w, 6);
    }
    for (int b = 0; b < m->nb; ++b) {
        real Ia[6], Iv[6], x[6];
        inertia_apply(w, w->I[b], w->ab[b], Ia);
        inertia_apply(w, w->I[b], w->vb[b], Iv);
        crf(w, w->vb[b], Iv, x);
        for (int k = 0; k < 6; ++k) w->f[b][k] = Ia[k] + x[k];
        FL(w, 6);
    }
    for (int b = m->nb - 1; b >= 1; --b) {
        int p = m->parent[b];
        cb[w->dof0 + b - 1] = sdot(w, w->S[b], w->f[b]);
        for (int k = 0; k < 6; ++k) w->f[p][k] += w->f[b][k];
        FL(w, 6);
    }
    if (!m->root_fixed) {
        real nb_[3];
        mattvec(w, w->R[0], w->f[0], nb_);
        cb[0] = w->f[0][3]; cb[1] = w->f[0][4]; cb[2] = w->f[0][5];
        cb[3] = nb_[0]; cb[4] = nb_[1]; cb[5] = nb_[2];
    }
}

/* ---------------------------------------------------------------- CRBA
 * Composite inertias summed leaf to root, then M_ij = S_i . (Ic_j S_j) along
 * the ancestor chain (Featherstone 2008, Table 6.2).  In world axes about O
 * no transform is needed between bodies. */
static void root_column(const orc_model* m, work* w, int k, real* S) {
    (void)m;
    memset(S, 0, 6 * sizeof(real));
    if (k < 3) S[3 + k] = 1.0;
    else col(w->R[0], k - 3, S);
}

static void crba(work* w, const orc_model* m, const orc_params* prm, real* M) {
    w->phase = ORC_PH_CRBA;
    int nv = w->nv;
    memset(M, 0, sizeof(real) * nv * nv);
    for (int b = 0; b < m->nb; ++b) memcpy(w->Ic[b], w->I[b], 10 * sizeof(real));
    for (int b = m->nb - 1; b >= 1; --b) {
        int p = m->parent[b];
        for (int k = 0; k < 10; ++k) w->Ic[p][k] += w->Ic[b][k];
        FL(w, 10);
    }
    for (int b = 1; b < m->nb; ++b) {
        int i = w->dof0 + b - 1;
        real F[6];
        inertia_apply(w, w->Ic[b], w->S[b], F);
        M[i * nv + i] = sdot(w, w->S[b], F) + prm->armature;
        FL(w, 1);
        for (int j = m->parent[b]; j > 0; j = m->parent[j]) {
            int jj = w->dof0 + j - 1;
            real x = sdot(w, w->S[j], F);
            M[jj * nv + i] = x;
            M[i * nv + jj] = x;
        }
        if (!m->root_fixed) {
            real Sr[6];
            for (int k = 0; k < 6; ++k) {
                root_column(m, w, k, Sr);
                real x = (k < 3) ? F[3 + k] : dot3(w, Sr, F);
                M[k * nv + i] = x;
                M[i * nv + k] = x;
            }
        }
    }
    if (!m->root_fixed) {
        for (int k = 0; k < 6; ++k) {
            real Sk[6], F[6], Sl[6];
            root_column(m, w, k, Sk);
            inertia_apply(w, w->Ic[0], Sk, F);
            for (int l = 0; l < 6; ++l) {
                root_column(m, w, l, Sl);
                M[l * nv + k] = sdot(w, Sl, F);
            }
        }
    }
}

/* ------------------------------------------------------------ Cholesky */
static int cholesky(work* w, int n, const real* M, real* L) {
    memset(L, 0, sizeof(real) * n * n);
    for (int j = 0; j < n; ++j) {
        real s = M[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        FL(w, 2 * j);
        if (!(s > 0.0)) return -1;
        real d = sqrt(s);
        L[j * n + j] = d;
        FL(w, 1);
        for (int i = j + 1; i < n; ++i) {
            real t = M[i * n + j];
            for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / d;
            FL(w, 2 * j + 1);
        }
    }
    return 0;
}

static void solve_lower(work* w, int n, const real* L, const real* b, real* y) {
    for (int i = 0; i < n; ++i) {
        real t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
        y[i] = t / L[i * n + i];
        FL(w, 2 * i + 1);
    }
}

static void solve_upper(work* w, int n, const real* L, const real* y, real* x) {
    for (int i = n - 1; i >= 0; --i) {
        real t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
        FL(w, 2 * (n - 1 - i) + 1);
    }
}

static void chol_solve(work* w, int n, const real* L, const real* b, real* x) {
    real y[ORC_MAXV];
    solve_lower(w, n, L, b, y);
    solve_upper(w, n, L, y, x);
}

/* ------------------------------------------------------------ contacts */
static void cand_add(orc_contact_list* cl, int a, int b, const real* p, const real* n, real d) {
    if (cl->n >= ORC_MAXCAND) return;
    int k = cl->n++;
    cl->a[k] = a; cl->b[k] = b;
    memcpy(cl->p[k], p, 3 * sizeof(real));
    memcpy(cl->nrm[k], n, 3 * sizeof(real));
    cl->depth[k] = d;
}

/* box/plane: every box vertex below z = 0 is a contact, vertex order k = 0..7
 * with bit 0 -> x sign, bit 1 -> y sign, bit 2 -> z sign (set = +). */
static void plane_contacts(work* w, const orc_model* m) {
    static const real up[3] = {0.0, 0.0, 1.0};
    for (int b = (m->root_fixed ? 1 : 0); b < m->nb; ++b) {
        if (m->geom[b] == ORC_GEOM_SPHERE) {
            /* sphere/plane: the lowest point of the sphere, if below z = 0 */
            real r = m->half[b][0];
            real pw[3] = {w->O[0] + w->c[b][0], w->O[1] + w->c[b][1], w->O[2] + w->c[b][2] - r};
            FL(w, 4);
            if ((pw[2] < 0.0) != decide(w, pw[2])) cand_add(&w->cand, b, -1, pw, up, -pw[2]);
            continue;
        }
        for (int k = 0; k < 8; ++k) {
            real lv[3], t[3], pw[3];
            for (int i = 0; i < 3; ++i) lv[i] = m->com[b][i] + (((k >> i) & 1) ? 1.0 : -1.0) * m->half[b][i];
            FL(w, 6);
            matvec(w, w->R[b], lv, t);
            for (int i = 0; i < 3; ++i) pw[i] = w->O[i] + w->r[b][i] + t[i];
            FL(w, 6);
            if ((pw[2] < 0.0) != decide(w, pw[2])) cand_add(&w->cand, b, -1, pw, up, -pw[2]);
        }
    }
}

/* Separating-axis test between two boxes and contact points.
 * Axes 0..2: faces of A, 3..5: faces of B, 6..14: A_i x B_j (6 + 3i + j).
 * Minimum-overlap axis, ties to the lowest index, with a face preferred unless
 * the best edge overlap is below 0.95 x the best face overlap.
 * Normals point from B (higher body index) towards A. */
static void box_box(work* w, const orc_model* m, int ia, int ib) {
    w->narrow++;
    real Ax[3][3], Bx[3][3];
    for (int k = 0; k < 3; ++k) { col(w->R[ia], k, Ax[k]); col(w->R[ib], k, Bx[k]); }
    const real* hA = m->half[ia];
    const real* hB = m->half[ib];
    real D[3];
    for (int k = 0; k < 3; ++k) D[k] = w->c[ib][k] - w->c[ia][k];
    FL(w, 3);
    real ov[15], Lx[15][3];
    int valid[15];
    real min_ov = 1e300;
    for (int e = 0; e < 15; ++e) {
        real L[3];
        valid[e] = 1;
        if (e < 3) memcpy(L, Ax[e], sizeof L);
        else if (e < 6) memcpy(L, Bx[e - 3], sizeof L);
        else {
            int i = (e - 6) / 3, j = (e - 6) % 3;
            cross3(w, Ax[i], Bx[j], L);
            real nl = sqrt(dot3(w, L, L));
            FL(w, 1);
            if (nl < 1e-6) { valid[e] = 0; ov[e] = 1e300; continue; }
            for (int k = 0; k < 3; ++k) L[k] /= nl;
            FL(w, 3);
        }
        real rA = 0.0, rB = 0.0;
        for (int k = 0; k < 3; ++k) {
            rA += hA[k] * fabs(dot3(w, Ax[k], L));
            rB += hB[k] * fabs(dot3(w, Bx[k], L));
        }
        FL(w, 12);
        ov[e] = rA + rB - fabs(dot3(w, D, L));
        FL(w, 3);
        memcpy(Lx[e], L, sizeof L);
        if (ov[e] < min_ov) min_ov = ov[e];
    }
    if ((min_ov <= 0.0) != decide(w, min_ov)) return;
    int bf = 0, be = -1;
    for (int e = 1; e < 6; ++e) if (ov[e] < ov[bf]) bf = e;
    for (int e = 6; e < 15; ++e) if (valid[e] && (be < 0 || ov[e] < ov[be])) be = e;
    /* margins of the axis choice (a reversed near tie takes the runner-up) */
    int fa = -1, ea = -1, fe = 0;
    for (int e = 0; e < 6; ++e)
        if (e != bf && decide(w, ov[e] - ov[bf]) && fa < 0) fa = e;
    if (be >= 0) {
        for (int e = 6; e < 15; ++e)
            if (valid[e] && e != be && decide(w, ov[e] - ov[be]) && ea < 0) ea = e;
        if (fa >= 0) bf = fa;
        if (ea >= 0) be = ea;
        fe = decide(w, ov[be] - 0.95 * ov[bf]);
        FL(w, 2);
    } else if (fa >= 0) {
        bf = fa;
    }
    int use_edge = be >= 0 && ((ov[be] < 0.95 * ov[bf]) != fe);
    if (!use_edge) {
        /* reference face from the owner of the axis, incident face on the other */
        int ref_is_A = bf < 3;
        int ri = ref_is_A ? bf : bf - 3;
        real (*Rx)[3] = ref_is_A ? Ax : Bx;
        real (*Ix)[3] = ref_is_A ? Bx : Ax;
        const real* hR = ref_is_A ? hA : hB;
        const real* hI = ref_is_A ? hB : hA;
        const real* cR = ref_is_A ? w->c[ia] : w->c[ib];
        const real* cI = ref_is_A ? w->c[ib] : w->c[ia];
        real toI[3];
        for (int k = 0; k < 3; ++k) toI[k] = cI[k] - cR[k];
        FL(w, 3);
        real sgn = dot3(w, toI, Rx[ri]) >= 0.0 ? 1.0 : -1.0;
        real nref[3] = {sgn * Rx[ri][0], sgn * Rx[ri][1], sgn * Rx[ri][2]};
        FL(w, 3);
        /* incident face: box face most anti-parallel to nref */
        real dd[3];
        int ki = 0;
        for (int k = 0; k < 3; ++k) dd[k] = dot3(w, Ix[k], nref);
        for (int k = 1; k < 3; ++k) if (fabs(dd[k]) > fabs(dd[ki])) ki = k;
        int ka = -1;
        for (int k = 0; k < 3; ++k)
            if (k != ki && decide(w, (fabs(dd[ki]) - fabs(dd[k])) * 0.05) && ka < 0) ka = k;
        if (ka >= 0) ki = ka;
        real si = dd[ki] > 0.0 ? -1.0 : 1.0;
        int k1 = (ki + 1) % 3, k2 = (ki + 2) % 3;
        if (k1 > k2) { int t = k1; k1 = k2; k2 = t; }
        real fc[3];
        for (int k = 0; k < 3; ++k) fc[k] = cI[k] + si * hI[ki] * Ix[ki][k];
        FL(w, 9);
        real poly[8][3], tmp[8][3];
        int np = 4;
        static const real s1[4] = {1, -1, -1, 1}, s2[4] = {1, 1, -1, -1};
        for (int v = 0; v < 4; ++v)
            for (int k = 0; k < 3; ++k)
                poly[v][k] = fc[k] + s1[v] * hI[k1] * Ix[k1][k] + s2[v] * hI[k2] * Ix[k2][k];
        FL(w, 4 * 3 * 6);
        /* clip against the reference face's side planes */
        int u1 = (ri + 1) % 3, u2 = (ri + 2) % 3;
        if (u1 > u2) { int t = u1; u1 = u2; u2 = t; }
        int pa[4] = {u1, u1, u2, u2};
        real ps[4] = {1.0, -1.0, 1.0, -1.0};
        for (int pl = 0; pl < 4 && np > 0; ++pl) {
            const real* u = Rx[pa[pl]];
            real e = hR[pa[pl]];
            /* side of every vertex: inside (-1), on the plane (0: within
               ORC_CLIP_ON of it) or outside (+1); vertices inside or on are
               kept, and a crossing point only joins an inside vertex to an
               outside one.  (An edge lying on the plane -- bricks touching on
               a lattice -- is then kept whole instead of cut at a point that
               rounding alone would place.) */
            real dist[8];
            int side[8];
            for (int v = 0; v < np; ++v) {
                real rel[3] = {poly[v][0] - cR[0], poly[v][1] - cR[1], poly[v][2] - cR[2]};
                FL(w, 3);
                dist[v] = ps[pl] * dot3(w, rel, u) - e;
                FL(w, 2);
                real ad = dist[v] < 0.0 ? -dist[v] : dist[v];
                int on = (ad <= ORC_CLIP_ON) != decide(w, ad - ORC_CLIP_ON);
                side[v] = on ? 0 : (dist[v] < 0.0 ? -1 : 1);
            }
            int no = 0;
            for (int v = 0; v < np; ++v) {
                int nx = (v + 1) % np;
                int in_v = side[v] <= 0;
                /* a convex quad gains at most one vertex per plane (<= 8); rounding
                   can only add spurious crossings, which are dropped past 8 */
                if (in_v && no < 8) { memcpy(tmp[no], poly[v], sizeof tmp[0]); ++no; }
                if (side[v] * side[nx] == -1 && no < 8) {
                    real t = dist[v] / (dist[v] - dist[nx]);
                    for (int k = 0; k < 3; ++k) tmp[no][k] = poly[v][k] + t * (poly[nx][k] - poly[v][k]);
                    FL(w, 2 + 9);
                    ++no;
                }
            }
            np = no;
            memcpy(poly, tmp, sizeof(real) * 3 * (size_t)np);
        }
        real nrm[3];
        for (int k = 0; k < 3; ++k) nrm[k] = ref_is_A ? -nref[k] : nref[k];
        for (int v = 0; v < np; ++v) {
            real rel[3] = {poly[v][0] - cR[0], poly[v][1] - cR[1], poly[v][2] - cR[2]};
            FL(w, 3);
            real depth = hR[ri] - dot3(w, rel, nref);
            FL(w, 1);
            if ((depth > 0.0) != decide(w, depth)) {
                real pw[3] = {poly[v][0] + w->O[0], poly[v][1] + w->O[1], poly[v][2] + w->O[2]};
                FL(w, 3);
                cand_add(&w->cand, ia, ib, pw, nrm, depth);
            }
        }
    } else {
        int i = (be - 6) / 3, j = (be - 6) % 3;
        real L[3];
        memcpy(L, Lx[be], sizeof L);
        if (dot3(w, D, L) < 0.0) { L[0] = -L[0]; L[1] = -L[1]; L[2] = -L[2]; }
        real PA[3], PB[3];
        for (int k = 0; k < 3; ++k) { PA[k] = w->c[ia][k]; PB[k] = w->c[ib][k]; }
        for (int k = 0; k < 3; ++k) {
            if (k != i) {
                real d = dot3(w, Ax[k], L);
                real s = ((d >= 0.0) != decide(w, d * hA[k])) ? hA[k] : -hA[k];
                for (int t = 0; t < 3; ++t) PA[t] += s * Ax[k][t];
                FL(w, 6);
            }
            if (k != j) {
                real d = dot3(w, Bx[k], L);
                real s = ((d >= 0.0) != decide(w, d * hB[k])) ? hB[k] : -hB[k];
                for (int t = 0; t < 3; ++t) PB[t] -= s * Bx[k][t];
                FL(w, 6);
            }
        }
        /* closest points of the lines PA + s Ax_i and PB + t Bx_j, clamped */
        real wv[3] = {PA[0] - PB[0], PA[1] - PB[1], PA[2] - PB[2]};
        FL(w, 3);
        real bb = dot3(w, Ax[i], Bx[j]);
        real dd = dot3(w, Ax[i], wv);
        real ee = dot3(w, Bx[j], wv);
        real den = 1.0 - bb * bb;
        real s = (bb * ee - dd) / den;
        real t = (ee - bb * dd) / den;
        FL(w, 2 + 3 + 3);
        if (s > hA[i]) s = hA[i];
        if (s < -hA[i]) s = -hA[i];
        if (t > hB[j]) t = hB[j];
        if (t < -hB[j]) t = -hB[j];
        FL(w, 4);
        real pw[3], nrm[3] = {-L[0], -L[1], -L[2]};
        for (int k = 0; k < 3; ++k)
            pw[k] = 0.5 * ((PA[k] + s * Ax[i][k]) + (PB[k] + t * Bx[j][k])) + w->O[k];
        FL(w, 3 * 7);
        cand_add(&w->cand, ia, ib, pw, nrm, ov[be]);
    }
}

/* Sphere/sphere and sphere/box, one contact at most.  The point is midway
 * between the two surfaces' deepest points along the normal; normals point
 * from body ib (higher index) towards body ia.
 *   sphere/sphere: n along the centre difference, depth r_a + r_b - |d|;
 *   sphere/box: Q = the box point closest to the sphere centre C (C clamped
 *     to the box in box axes); C outside: n = (C - Q) / |C - Q|, depth
 *     r - |C - Q|; C inside: n = the normal of the nearest face (smallest
 *     h_k - |C_k|, ties to the lowest k), depth r + h_k - |C_k|. */
static void sphere_pair(work* w, const orc_model* m, int ia, int ib) {
    w->narrow++;
    int sa = m->geom[ia] == ORC_GEOM_SPHERE, sb = m->geom[ib] == ORC_GEOM_SPHERE;
    real p[3], n[3];
    if (sa && sb) {
        real ra = m->half[ia][0], rb = m->half[ib][0];
        real d[3] = {w->c[ia][0] - w->c[ib][0], w->c[ia][1] - w->c[ib][1], w->c[ia][2] - w->c[ib][2]};
        real dist = sqrt(dot3(w, d, d));
        real depth = ra + rb - dist;
        FL(w, 3 + 1 + 2);
        if (((depth > 0.0) == decide(w, depth)) || !(dist > 0.0)) return;
        for (int k = 0; k < 3; ++k) {
            n[k] = d[k] / dist;
            p[k] = w->O[k] + 0.5 * ((w->c[ia][k] - ra * n[k]) + (w->c[ib][k] + rb * n[k]));
        }
        FL(w, 3 * 8);
        cand_add(&w->cand, ia, ib, p, n, depth);
        return;
    }
    int is = sa ? ia : ib, ix = sa ? ib : ia;  /* the sphere and the box */
    real r = m->half[is][0];
    const real* h = m->half[ix];
    const real* R = w->R[ix];
    real D[3] = {w->c[is][0] - w->c[ix][0], w->c[is][1] - w->c[ix][1], w->c[is][2] - w->c[ix][2]};
    real l[3], q[3], e[3];
    for (int k = 0; k < 3; ++k) {
        l[k] = R[k] * D[0] + R[3 + k] * D[1] + R[6 + k] * D[2];  /* R^T D: box axes */
        q[k] = l[k] > h[k] ? h[k] : (l[k] < -h[k] ? -h[k] : l[k]);
        e[k] = l[k] - q[k];
    }
    FL(w, 3 + 3 * 5 + 3);
    real e2 = dot3(w, e, e);
    real nl[3], pl[3], depth;
    if (e2 > 0.0) {
        real dist = sqrt(e2);
        depth = r - dist;
        FL(w, 2);
        note_margin(w, dist);
        if ((depth > 0.0) == decide(w, depth)) return;
        for (int k = 0; k < 3; ++k) { nl[k] = e[k] / dist; pl[k] = q[k] - 0.5 * depth * nl[k]; }
        FL(w, 3 * 4);
    } else {
        int kk = 0;
        real pen = h[0] - fabs(l[0]);
        for (int k = 1; k < 3; ++k) {
            real pk = h[k] - fabs(l[k]);
            if (pk < pen) { pen = pk; kk = k; }
        }
        FL(w, 3 * 2);
        int ka = -1;
        for (int k = 0; k < 3; ++k)
            if (k != kk && decide(w, (h[k] - fabs(l[k])) - pen) && ka < 0) ka = k;
        note_margin(w, h[kk] - pen);  /* distance of the centre from the surface */
        if (ka >= 0) {
            kk = ka;
            pen = h[kk] - fabs(l[kk]);
        }
        depth = r + pen;
        for (int k = 0; k < 3; ++k) nl[k] = 0.0;
        nl[kk] = l[kk] >= 0.0 ? 1.0 : -1.0;
        for (int k = 0; k < 3; ++k) pl[k] = l[k] + 0.5 * (pen - r) * nl[k];
        FL(w, 1 + 3 * 4);
    }
    /* to world; the box-to-sphere normal is flipped when the sphere is ib */
    real sg = is == ia ? 1.0 : -1.0;
    for (int k = 0; k < 3; ++k) {
        n[k] = sg * (R[3 * k] * nl[0] + R[3 * k + 1] * nl[1] + R[3 * k + 2] * nl[2]);
        p[k] = w->O[k] + w->c[ix][k] + (R[3 * k] * pl[0] + R[3 * k + 1] * pl[1] + R[3 * k + 2] * pl[2]);
    }
    FL(w, 3 * 6 + 3 * 7);
    cand_add(&w->cand, ia, ib, p, n, depth);
}

static int gen_contacts(work* w, const orc_model* m, const orc_params* prm) {
    w->phase = ORC_PH_CONTACT;
    w->cand.n = 0;
    if (prm->ground) plane_contacts(w, m);
    if (prm->box_box) {
        real rad[ORC_MAXB];
        for (int b = 0; b < m->nb; ++b) {
            if (m->geom[b] == ORC_GEOM_SPHERE) {
                rad[b] = m->half[b][0];
            } else {
                rad[b] = sqrt(m->half[b][0] * m->half[b][0] + m->half[b][1] * m->half[b][1] +
                              m->half[b][2] * m->half[b][2]);
                FL(w, 6);
            }
        }
        for (int a = 0; a < m->nb; ++a)
            for (int b = a + 1; b < m->nb; ++b) {
                if (m->parent[b] == a || ((m->exclude[a] >> b) & 1u)) continue;
                w->broad++;
                real d[3] = {w->c[b][0] - w->c[a][0], w->c[b][1] - w->c[a][1], w->c[b][2] - w->c[a][2]};
                real rr = rad[a] + rad[b];
                FL(w, 4 + 5 + 2);
                if (dot3(w, d, d) <= rr * rr) {
                    if (m->geom[a] == ORC_GEOM_BOX && m->geom[b] == ORC_GEOM_BOX) box_box(w, m, a, b);
                    else sphere_pair(w, m, a, b);
                }
            }
    }
    /* keep the contact_cap deepest, ties by list order, list order kept */
    int cap = prm->contact_cap;
    int st = 0;
    kept_list* K = &w->con;
    K->n = 0;
    int n = w->cand.n;
    if (n > cap) {
        st |= ORC_ST_OVERFLOW;
        real d_last = 0.0, d_first_out = 0.0;
        static _Thread_local int rank_of[ORC_MAXCAND];
        for (int i = 0; i < n; ++i) {
            int rank = 0;
            for (int j = 0; j < n; ++j)
                if (w->cand.depth[j] > w->cand.depth[i] || (w->cand.depth[j] == w->cand.depth[i] && j < i)) ++rank;
            if (rank == cap - 1) d_last = w->cand.depth[i];
            if (rank == cap) d_first_out = w->cand.depth[i];
            rank_of[i] = rank;
        }
        /* gap between the last kept and the first dropped depth (reversed:
           the two trade places) */
        int swap = decide(w, d_last - d_first_out);
        for (int i = 0; i < n; ++i) {
            int rank = rank_of[i];
            if (swap && (rank == cap - 1 || rank == cap)) rank = rank == cap ? cap - 1 : cap;
            if (rank < cap) {
                int k = K->n++;
                K->a[k] = w->cand.a[i]; K->b[k] = w->cand.b[i];
                memcpy(K->p[k], w->cand.p[i], sizeof K->p[0]);
                memcpy(K->nrm[k], w->cand.nrm[i], sizeof K->nrm[0]);
                K->depth[k] = w->cand.depth[i];
            }
        }
        FL(w, (real)n * n);
    } else {
        for (int i = 0; i < n; ++i) {
            int k = K->n++;
            K->a[k] = w->cand.a[i]; K->b[k] = w->cand.b[i];
            memcpy(K->p[k], w->cand.p[i], sizeof K->p[0]);
            memcpy(K->nrm[k], w->cand.nrm[i], sizeof K->nrm[0]);
            K->depth[k] = w->cand.depth[i];
        }
    }
    return st;
}

/* orthonormal tangents from a unit normal (Duff et al. 2017, JCGT 6(1)) */
static void tangent_basis(work* w, const real* n, real* t1, real* t2) {
    real s = n[2] >= 0.0 ? 1.0 : -1.0;
    real a = -1.0 / (s + n[2]);
    real b = n[0] * n[1] * a;
    t1[0] = 1.0 + s * n[0] * n[0] * a; t1[1] = s * b; t1[2] = -s * n[0];
    t2[0] = b; t2[1] = s + n[1] * n[1] * a; t2[2] = -n[1];
    FL(w, 2 + 2 + 4 + 2 + 1 + 3 + 1);
}

/* Tangents of a body-pair contact: Duff's basis built in the fixed frame G
 * whose rows are g1 = (-sqrt(2/3), sqrt(1/3), 0), g2 = (-1/sqrt6, -1/sqrt3,
 * 1/sqrt2), g3 = (1, sqrt2, sqrt3)/sqrt6, then turned back (reading: the
 * basis jumps where (G n)_z changes sign, on normals orthogonal to g3, instead
 * of on the horizontal normals lattice-built bricks side by side produce;
 * the Gauss-Seidel result depends on the basis).  Ground contacts keep
 * tangent_basis: x and y. */
static void pair_tangent_basis(work* w, const real* n, real* t1, real* t2) {
    const real r2 = sqrt(2.0), r3 = sqrt(3.0), r6 = sqrt(6.0);
    const real G[3][3] = {{-r2 / r3, 1.0 / r3, 0.0}, {-1.0 / r6, -1.0 / r3, 1.0 / r2}, {1.0 / r6, r2 / r6, r3 / r6}};
    real m[3], u1[3], u2[3];
    for (int i = 0; i < 3; ++i) m[i] = G[i][0] * n[0] + G[i][1] * n[1] + G[i][2] * n[2];
    FL(w, 15);
    tangent_basis(w, m, u1, u2);
    for (int k = 0; k < 3; ++k) {
        t1[k] = G[0][k] * u1[0] + G[1][k] * u1[1] + G[2][k] * u1[2];
        t2[k] = G[0][k] * u2[0] + G[1][k] * u2[1] + G[2][k] * u2[2];
    }
    FL(w, 30);
}

/* is body k (>= 1) the body x or one of its ancestors? */
static int on_path(const orc_model* m, int x, int k) {
    for (int y = x; y > 0; y = m->parent[y]) if (y == k) return 1;
    return 0;
}

/* Jacobian row of the relative velocity of body a w.r.t. body b at world
 * point pw along direction d (b = -1: ground). */
static void jac_row(work* w, const orc_model* m, int a, int b, const real* pw, const real* d, real* J) {
    int nv = w->nv;
    memset(J, 0, sizeof(real) * nv);
    real rp[3] = {pw[0] - w->O[0], pw[1] - w->O[1], pw[2] - w->O[2]};
    FL(w, 3);
    real rxd[3];
    cross3(w, rp, d, rxd);
    if (!m->root_fixed) {
        real s = (a >= 0 ? 1.0 : 0.0) - (b >= 0 ? 1.0 : 0.0);
        if (s != 0.0) {
            real e[3];
            for (int i = 0; i < 3; ++i) {
                J[i] = s * d[i];
                col(w->R[0], i, e);
                J[3 + i] = s * dot3(w, e, rxd);
            }
            FL(w, 6);
        }
    }
    for (int k = 1; k < m->nb; ++k) {
        real s = (a >= 0 ? on_path(m, a, k) : 0) - (b >= 0 ? on_path(m, b, k) : 0);
        if (s == 0.0) continue;
        /* axis_k x (p - r_k) . d = axis_k . ((p - r_k) x d) */
        real rel[3] = {rp[0] - w->r[k][0], rp[1] - w->r[k][1], rp[2] - w->r[k][2]};
        real x[3];
        FL(w, 3);
        cross3(w, rel, d, x);
        J[w->dof0 + k - 1] = s * dot3(w, w->S[k], x);
        FL(w, 1);
    }
}

/* ------------------------------------------------------------- step */
static int step(work* w, const orc_model* m, const orc_params* prm, real* q, real* v, real* s,
                uint32_t* status, real* vfree_out, real* lam_out, int32_t* nc_out) {
    if (*status & (ORC_ST_NONFINITE | ORC_ST_CHOL)) return 0;
    setup(w, m);
    int nv = w->nv, nh = m->nb - 1;
    real dt = prm->dt;
    uint32_t st = 0;

    /* 1. CPG: s <- s + dt W s, W antisymmetric; PD torque to the targets */
    w->phase = ORC_PH_CPG;
    real sn[2 * ORC_MAXB];
    memset(w->tau, 0, sizeof w->tau);
    if (prm->actuate) {
        real ds[2 * ORC_MAXB];
        for (int i = 0; i < nh; ++i) {
            int b = i + 1;
            ds[2 * i] = m->w_int[b] * s[2 * i + 1];
            ds[2 * i + 1] = -m->w_int[b] * s[2 * i];
            FL(w, 2);
        }
        for (int i = 0; i < nh; ++i) {
            int b = i + 1, p = m->parent[b];
            if (p >= 1) {
                int j = p - 1;
                real wc = m->w_cpl[b];
                ds[2 * j] += wc * s[2 * i];
                ds[2 * i] -= wc * s[2 * j];
                FL(w, 4);
            }
        }
        for (int i = 0; i < 2 * nh; ++i) sn[i] = s[i] + dt * ds[i];
        FL(w, 4 * nh);
        for (int i = 0; i < nh; ++i) {
            real x = sn[2 * i];
            if (x > 1.0) x = 1.0;
            if (x < -1.0) x = -1.0;
            real target = prm->theta_max * x;
            real th = q[w->q0h + i], thd = v[w->dof0 + i];
            real t = prm->kp * (target - th) - prm->kd * thd;
            if (t > prm->tau_max) t = prm->tau_max;
            if (t < -prm->tau_max) t = -prm->tau_max;
            w->tau[w->dof0 + i] = t;
            FL(w, 2 + 1 + 4 + 2);
        }
    } else {
        for (int i = 0; i < 2 * nh; ++i) sn[i] = s[i];
    }

    /* 2-4. kinematics, bias forces, mass matrix */
    fk(w, m, q);
    motion_subspaces(w, m);
    w->phase = ORC_PH_RNEA;
    body_inertias(w, m);
    rnea(w, m, prm, v, w->cb);
    crba(w, m, prm, w->M);

    /* 5. Cholesky and the unconstrained velocity */
    w->phase = ORC_PH_CHOL;
    if (cholesky(w, nv, w->M, w->L) != 0) {
        *status |= ORC_ST_CHOL;
        return 0;
    }
    {
        real rhs[ORC_MAXV], acc[ORC_MAXV];
        for (int i = 0; i < nv; ++i) rhs[i] = w->tau[i] - w->cb[i];
        FL(w, nv);
        chol_solve(w, nv, w->L, rhs, acc);
        for (int i = 0; i < nv; ++i) w->vfree[i] = v[i] + dt * acc[i];
        FL(w, 2 * nv);
    }

    /* 6. contacts */
    st |= (uint32_t)gen_contacts(w, m, prm);
    int nc = w->con.n;

    /* 7. contact Jacobians, W = M^-1 J^T, diagonal of J M^-1 J^T */
    w->phase = ORC_PH_JAC;
    real omg = 2.0 * ORC_PI / prm->soft_tau;
    real kden = dt * omg * omg + 2.0 * prm->soft_zeta * omg;
    real erp = dt * omg * omg / kden;
    real kappa = 1.0 / (dt * kden);
    FL(w, 14);
    for (int k = 0; k < nc; ++k) {
        real t1[3], t2[3];
        const real* n = w->con.nrm[k];
        if (w->con.b[k] < 0) tangent_basis(w, n, t1, t2);
        else pair_tangent_basis(w, n, t1, t2);
        const real* dirs[3] = {n, t1, t2};
        for (int d = 0; d < 3; ++d) {
            int r = 3 * k + d;
            jac_row(w, m, w->con.a[k], w->con.b[k], w->con.p[k], dirs[d], w->J[r]);
            chol_solve(w, nv, w->L, w->J[r], w->Wm[r]);
            real a = 0.0;
            for (int i = 0; i < nv; ++i) a += w->J[r][i] * w->Wm[r][i];
            FL(w, 2 * nv);
            /* a row that no dof can move (J = 0, e.g. a tangent normal to the
               plane of a planar mechanism) carries no impulse: frozen at 0 */
            w->A[r] = ((a > ORC_AMIN) != decide(w, (a - ORC_AMIN) * 1e4)) ? a : 0.0;
            /* softness R = kappa A (mass-normalised CFM), floored: a row that the
               dofs can barely move (A -> 0 but above the freeze threshold) would
               otherwise take an impulse ~ 1 / A and inject ~ g^2 / (2 A) of
               kinetic energy; with R >= min_cfm a row's kinetic energy change
               is at most g^2 / (8 min_cfm) */
            w->Rs[r] = kappa * a > prm->min_cfm ? kappa * a : prm->min_cfm;
            if (d == 0) {
                /* penetration recovery speed, capped (ODE's maximum correcting velocity) */
                real tn = erp * w->con.depth[k] / dt;
                note_margin(w, (tn - prm->max_correct_vel) * dt / erp);
                w->tgt[r] = tn < prm->max_correct_vel ? tn : prm->max_correct_vel;
            } else {
                w->tgt[r] = 0.0;
            }
            FL(w, d == 0 ? 3 : 1);
            w->lam[r] = 0.0;
        }
    }

    /* 8. soft projected Gauss-Seidel, fixed sweeps, list order */
    w->phase = ORC_PH_PGS;
    real* vv = w->vnew;
    memcpy(vv, w->vfree, sizeof(real) * nv);
    for (int it = 0; it < prm->pgs_iters; ++it) {
        for (int k = 0; k < nc; ++k) {
            int rn = 3 * k, r1 = rn + 1, r2 = rn + 2;
            real jv = 0.0;
            for (int i = 0; i < nv; ++i) jv += w->J[rn][i] * vv[i];
            real g = jv - w->tgt[rn] + w->Rs[rn] * w->lam[rn];
            real ln = w->A[rn] > 0.0 ? w->lam[rn] - g / (w->A[rn] + w->Rs[rn]) : w->lam[rn];
            if (ln < 0.0) ln = 0.0;
            real dn = ln - w->lam[rn];
            for (int i = 0; i < nv; ++i) vv[i] += w->Wm[rn][i] * dn;
            w->lam[rn] = ln;
            FL(w, 4 * nv + 3 + 3 + 1 + 1);
            real j1 = 0.0, j2 = 0.0;
            for (int i = 0; i < nv; ++i) { j1 += w->J[r1][i] * vv[i]; j2 += w->J[r2][i] * vv[i]; }
            real l1 = w->A[r1] > 0.0 ? w->lam[r1] - (j1 + w->Rs[r1] * w->lam[r1]) / (w->A[r1] + w->Rs[r1]) : w->lam[r1];
            real l2 = w->A[r2] > 0.0 ? w->lam[r2] - (j2 + w->Rs[r2] * w->lam[r2]) / (w->A[r2] + w->Rs[r2]) : w->lam[r2];
            real lim = prm->mu * ln;
            real nt2 = l1 * l1 + l2 * l2;
            FL(w, 4 * nv + 10 + 1 + 3);
            if (nt2 > lim * lim) {
                real sc = lim / sqrt(nt2);
                l1 *= sc; l2 *= sc;
                FL(w, 5);
            }
            FL(w, 1);
            real d1 = l1 - w->lam[r1], d2 = l2 - w->lam[r2];
            for (int i = 0; i < nv; ++i) vv[i] += w->Wm[r1][i] * d1 + w->Wm[r2][i] * d2;
            w->lam[r1] = l1; w->lam[r2] = l2;
            FL(w, 2 + 4 * nv);
        }
    }

    /* 9. semi-implicit Euler on the configuration */
    w->phase = ORC_PH_INTEG;
    real qn[ORC_MAXQ];
    memcpy(qn, q, sizeof(real) * w->nq);
    if (!m->root_fixed) {
        for (int i = 0; i < 3; ++i) qn[i] = q[i] + dt * vv[i];
        FL(w, 6);
        const real* om = vv + 3;
        real nw = sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
        FL(w, 6);
        real dq[4] = {1.0, 0.0, 0.0, 0.0};
        if (nw >= 1e-12) {
            real ha = 0.5 * dt * nw;
            real sa = sin(ha) / nw;
            dq[0] = cos(ha);
            dq[1] = sa * om[0]; dq[2] = sa * om[1]; dq[3] = sa * om[2];
            FL(w, 2 + 2 + 1 + 3);
        }
        const real* a = q + 3;
        real r[4];
        r[0] = a[0] * dq[0] - a[1] * dq[1] - a[2] * dq[2] - a[3] * dq[3];
        r[1] = a[0] * dq[1] + a[1] * dq[0] + a[2] * dq[3] - a[3] * dq[2];
        r[2] = a[0] * dq[2] - a[1] * dq[3] + a[2] * dq[0] + a[3] * dq[1];
        r[3] = a[0] * dq[3] + a[1] * dq[2] - a[2] * dq[1] + a[3] * dq[0];
        real nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
        for (int i = 0; i < 4; ++i) qn[3 + i] = r[i] / nr;
        FL(w, 28 + 8 + 4);
    }
    for (int i = 0; i < nh; ++i) qn[w->q0h + i] = q[w->q0h + i] + dt * vv[w->dof0 + i];
    FL(w, 2 * nh);

    /* non-finite state freezes the variant (state left as it was) */
    int bad = 0;
    for (int i = 0; i < w->nq; ++i) if (!isfinite(qn[i])) bad = 1;
    for (int i = 0; i < nv; ++i) if (!isfinite(vv[i])) bad = 1;
    for (int i = 0; i < 2 * nh; ++i) if (!isfinite(sn[i])) bad = 1;
    if (vfree_out) memcpy(vfree_out, w->vfree, sizeof(real) * nv);
    if (lam_out) memcpy(lam_out, w->lam, sizeof(real) * 3 * nc);
    if (nc_out) *nc_out = nc;
    if (bad) {
        *status |= ORC_ST_NONFINITE | st;
        return nc;
    }
    memcpy(q, qn, sizeof(real) * w->nq);
    memcpy(v, vv, sizeof(real) * nv);
    memcpy(s, sn, sizeof(real) * 2 * nh);
    *status |= st;
    return nc;
}

static work* work_new(void) {
    work* w = (work*)calloc(1, sizeof(work));
    return w;
}

int orc_run(const orc_model* m, const orc_params* prm, int nsteps, real* q, real* v, real* s,
            uint32_t* status, orc_stats* st) {
    work* w = work_new();
    if (!w) return -1;
    for (int t = 0; t < nsteps; ++t) {
        w->margin = 1e300;
        w->narrow = w->broad = 0;
        uint32_t before = *status;
        int nc = step(w, m, prm, q, v, s, status, NULL, NULL, NULL);
        if (st) {
            st->contacts += nc;
            st->narrow_pairs += w->narrow;
            st->broad_pairs += w->broad;
            if (st->steps == 0 || w->margin < st->margin) st->margin = w->margin;
            if ((*status & ORC_ST_OVERFLOW) && !(before & ORC_ST_OVERFLOW)) st->overflow_steps++;
            st->steps++;
        }
    }
    if (st)
        for (int k = 0; k < ORC_NPHASE; ++k) st->flops[k] += w->flops[k];
    free(w);
    return 0;
}

int orc_step_detail(const orc_model* m, const orc_params* prm, real* q, real* v, real* s,
                    uint32_t* status, real* vfree_out, real* lambda_out, int32_t* nc_out) {
    work* w = work_new();
    if (!w) return -1;
    w->margin = 1e300;
    step(w, m, prm, q, v, s, status, vfree_out, lambda_out, nc_out);
    free(w);
    return 0;
}

int orc_step_flip(const orc_model* m, const orc_params* prm, real* q, real* v, real* s, uint32_t* status,
                  double band, const int32_t* flip, int32_t nflip, int32_t* near_out, int32_t* nnear_out,
                  double* margin_out) {
    if (nflip < 0 || nflip > ORC_MAXNEAR || (nflip > 0 && !flip)) return -1;
    work* w = work_new();
    if (!w) return -1;
    w->margin = 1e300;
    w->band = band;
    w->nflip = nflip;
    for (int k = 0; k < nflip; ++k) w->flip[k] = flip[k];
    step(w, m, prm, q, v, s, status, NULL, NULL, NULL);
    if (near_out)
        for (int k = 0; k < w->nnear && k < ORC_MAXNEAR; ++k) near_out[k] = w->near[k];
    if (nnear_out) *nnear_out = w->nnear;
    if (margin_out) *margin_out = w->margin;
    free(w);
    return 0;
}

void orc_fk(const orc_model* m, const real* q, real* R, real* p, real* c) {
    work* w = work_new();
    setup(w, m);
    fk(w, m, q);
    for (int b = 0; b < m->nb; ++b) {
        if (R) memcpy(R + 9 * b, w->R[b], 9 * sizeof(real));
        for (int k = 0; k < 3; ++k) {
            if (p) p[3 * b + k] = w->O[k] + w->r[b][k];
            if (c) c[3 * b + k] = w->O[k] + w->c[b][k];
        }
    }
    free(w);
}

void orc_mass_matrix(const orc_model* m, const orc_params* prm, const real* q, real* M) {
    work* w = work_new();
    setup(w, m);
    fk(w, m, q);
    motion_subspaces(w, m);
    body_inertias(w, m);
    crba(w, m, prm, M);
    free(w);
}

void orc_bias(const orc_model* m, const orc_params* prm, const real* q, const real* v, real* c) {
    work* w = work_new();
    setup(w, m);
    fk(w, m, q);
    motion_subspaces(w, m);
    body_inertias(w, m);
    rnea(w, m, prm, v, c);
    free(w);
}

int orc_cholesky(int n, const real* M, real* L) {
    work* w = work_new();
    int r = cholesky(w, n, M, L);
    free(w);
    return r;
}

static int contacts_of(const orc_model* m, const orc_params* prm, const real* q, double band,
                       const int32_t* flip, int32_t nflip, orc_contact_list* out, int32_t* near_out,
                       int32_t* nnear_out, double* margin_out) {
    if (nflip < 0 || nflip > ORC_MAXNEAR || (nflip > 0 && !flip)) return -1;
    work* w = work_new();
    if (!w) return -1;
    setup(w, m);
    w->margin = 1e300;
    w->band = band;
    w->nflip = nflip;
    for (int k = 0; k < nflip; ++k) w->flip[k] = flip[k];
    fk(w, m, q);
    int st = gen_contacts(w, m, prm);
    out->n = w->con.n;
    for (int k = 0; k < w->con.n; ++k) {
        out->a[k] = w->con.a[k];
        out->b[k] = w->con.b[k];
        memcpy(out->p[k], w->con.p[k], sizeof out->p[0]);
        memcpy(out->nrm[k], w->con.nrm[k], sizeof out->nrm[0]);
        out->depth[k] = w->con.depth[k];
    }
    if (near_out)
        for (int k = 0; k < w->nnear && k < ORC_MAXNEAR; ++k) near_out[k] = w->near[k];
    if (nnear_out) *nnear_out = w->nnear;
    if (margin_out) *margin_out = w->margin;
    free(w);
    return st;
}

int orc_contacts(const orc_model* m, const orc_params* prm, const real* q, orc_contact_list* out,
                 real* margin) {
    double mg = 0.0;
    int st = contacts_of(m, prm, q, 0.0, NULL, 0, out, NULL, NULL, &mg);
    if (margin) *margin = (real)mg;
    return st;
}

int orc_contacts_flip(const orc_model* m, const orc_params* prm, const real* q, double band,
                      const int32_t* flip, int32_t nflip, orc_contact_list* out, int32_t* near_out,
                      int32_t* nnear_out, double* margin_out) {
    return contacts_of(m, prm, q, band, flip, nflip, out, near_out, nnear_out, margin_out);
}

/* ------------------------------------------------ threads over variants */
typedef struct {
    const orc_model* m;
    const orc_params* prm;
    int nsteps, first, last;
    real *q, *v, *s;
    int qs, vs, ss;
    uint32_t* status;
    orc_stats st;
} job;

static void* job_main(void* arg) {
    job* j = (job*)arg;
    memset(&j->st, 0, sizeof j->st);
    j->st.margin = 1e300;
    for (int i = j->first; i < j->last; ++i) {
        orc_stats one;
        memset(&one, 0, sizeof one);
        one.margin = 1e300;
        orc_run(j->m + i, j->prm, j->nsteps, j->q + (size_t)i * j->qs, j->v + (size_t)i * j->vs,
                j->s + (size_t)i * j->ss, j->status + i, &one);
        for (int k = 0; k < ORC_NPHASE; ++k) j->st.flops[k] += one.flops[k];
        j->st.contacts += one.contacts;
        j->st.narrow_pairs += one.narrow_pairs;
        j->st.broad_pairs += one.broad_pairs;
        if (one.margin < j->st.margin) j->st.margin = one.margin;
        j->st.overflow_steps += one.overflow_steps;
        j->st.steps += one.steps;
    }
    return NULL;
}

int orc_run_many(const orc_model* m, int nvar, const orc_params* prm, int nsteps, real* q, int q_stride,
                 real* v, int v_stride, real* s, int s_stride, uint32_t* status, orc_stats* st,
                 int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nvar) nthreads = nvar > 0 ? nvar : 1;
    job* jobs = (job*)calloc((size_t)nthreads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].m = m; jobs[t].prm = prm; jobs[t].nsteps = nsteps;
        jobs[t].first = (int)((long)nvar * t / nthreads);
        jobs[t].last = (int)((long)nvar * (t + 1) / nthreads);
        jobs[t].q = q; jobs[t].v = v; jobs[t].s = s;
        jobs[t].qs = q_stride; jobs[t].vs = v_stride; jobs[t].ss = s_stride;
        jobs[t].status = status;
        pthread_create(&th[t], NULL, job_main, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (st) {
        memset(st, 0, sizeof *st);
        st->margin = 1e300;
        for (int t = 0; t < nthreads; ++t) {
            for (int k = 0; k < ORC_NPHASE; ++k) st->flops[k] += jobs[t].st.flops[k];
            st->contacts += jobs[t].st.contacts;
            st->narrow_pairs += jobs[t].st.narrow_pairs;
            st->broad_pairs += jobs[t].st.broad_pairs;
            if (jobs[t].st.margin < st->margin) st->margin = jobs[t].st.margin;
            st->overflow_steps += jobs[t].st.overflow_steps;
            st->steps += jobs[t].st.steps;
        }
    }
    free(jobs);
    free(th);
    return 0;
}
