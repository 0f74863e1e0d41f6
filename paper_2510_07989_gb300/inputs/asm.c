/*
 * CPU FP64 assembly of the interaction matrices of the qHP TD-PMCHWT
 * (paper Section V-B) and of the static operators on the barycentric
 * refinement (paper Section III). Input generator: its matrices feed both the
 * CUDA MOT path and the oracle.
 *
 * Per medium (wave speed c) and lag k, with tau = k dt - R/c, R = |x - y|, and
 * RWG functions f_m (test, on triangle S) and f_n (source, on triangle R):
 *
 *   family A  (h_0 source basis, collocation at t = k dt; Section V-B-1):
 *     T_k = -(1/(4 pi c)) <<f_m . f_n  h_0'(tau) / R>>
 *     K_k =  (1/(4 pi))   <<(x-y).(f_m x f_n) [h_0'(tau)/(c R^2) + h_0(tau)/R^3]>>
 *   family Ah (T_max d/dt of the q_0 source basis, full T = T^s + T^h; V-B-2):
 *     T^_k = T_max [ -(1/(4 pi c)) <<f_m . f_n q_0''(tau)/R>>
 *                    -(c/(4 pi))   <<div f_m div f_n q_0(tau)/R>> ]
 *     K^_k = T_max (1/(4 pi)) <<(x-y).(f_m x f_n) [q_0''/(c R^2) + q_0'/R^3]>>
 *   family At ((1/T_max) d/dt^-1 of the p_0 source basis, T^s only; V-B-3):
 *     T~_k = (1/T_max) (-(1/(4 pi c))) <<f_m . f_n p_0(tau)/R>>
 *     K~_k = (1/T_max) (1/(4 pi)) <<(x-y).(f_m x f_n) [p_0/(c R^2) + P(tau)/R^3]>>
 *           with P = d/dt^-1 p_0 (0, ramp, then dt: the constant tail
 *           (dt/T_max) K_0 of the paper).
 *
 * The time bases are piecewise polynomials with knots at multiples of dt, so
 * every integrand is smooth between the spheres |x - y| = j c dt. The inner
 * (source) integral uses polar coordinates about the projection of the test
 * point on the source plane, split exactly at those spheres, with a sinh
 * substitution of the in-plane radius that removes the 1/R and 1/R^3 (near-)
 * singularities; the outer (test) integral uses a symmetric N_q-point rule.
 *
 * K~ is stored as an explicit lag window plus a constant tail (value, first lag)
 * per matrix entry. Lags of the At family at k >= k_max are dropped (the
 * explicit truncation the paper prescribes for Q^sl).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

typedef struct {
    double p[3][3];
    double n[3];
    double area;
    double cen[3];
    double diam;
} Tri;

/* ------------------------------------------------------------------ vectors */
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void sub3(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static inline void cross3(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double* a) { return sqrt(dot3(a, a)); }

static void make_tri(const double* V, const int* idx, Tri* t) {
    for (int i = 0; i < 3; i++)
        for (int d = 0; d < 3; d++) t->p[i][d] = V[3 * idx[i] + d];
    double e1[3], e2[3], c[3];
    sub3(t->p[1], t->p[0], e1);
    sub3(t->p[2], t->p[0], e2);
    cross3(e1, e2, c);
    double nc = norm3(c);
    t->area = 0.5 * nc;
    for (int d = 0; d < 3; d++) {
        t->n[d] = c[d] / nc;
        t->cen[d] = (t->p[0][d] + t->p[1][d] + t->p[2][d]) / 3.0;
    }
    double d01[3], d12[3], d20[3];
    sub3(t->p[1], t->p[0], d01);
    sub3(t->p[2], t->p[1], d12);
    sub3(t->p[0], t->p[2], d20);
    double a = norm3(d01), b = norm3(d12), cc = norm3(d20);
    t->diam = a > b ? (a > cc ? a : cc) : (b > cc ? b : cc);
}

/* Gauss-Legendre nodes/weights on [0, 1] (Newton on P_n). */
static void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; i++) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* Symmetric triangle rules (barycentric), weights summing to 1. */
static int tri_rule(int n, double* bary, double* w) {
    if (n == 1) {
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 1.0;
        return 1;
    }
    if (n == 3) {
        double a = 2.0 / 3.0, b = 1.0 / 6.0;
        double P[9] = {a, b, b, b, a, b, b, b, a};
        memcpy(bary, P, sizeof P);
        w[0] = w[1] = w[2] = 1.0 / 3.0;
        return 3;
    }
    if (n == 4) {
        double P[12] = {1. / 3, 1. / 3, 1. / 3, .6, .2, .2, .2, .6, .2, .2, .2, .6};
        memcpy(bary, P, sizeof P);
        w[0] = -27.0 / 48.0;
        w[1] = w[2] = w[3] = 25.0 / 48.0;
        return 4;
    }
    if (n == 6) {
        double a = 0.445948490915965, wa = 0.223381589678011;
        double b = 0.091576213509771, wb = 0.109951743655322;
        double P[18] = {a, a, 1 - 2 * a, a, 1 - 2 * a, a, 1 - 2 * a, a, a,
                        b, b, 1 - 2 * b, b, 1 - 2 * b, b, 1 - 2 * b, b, b};
        memcpy(bary, P, sizeof P);
        for (int i = 0; i < 3; i++) { w[i] = wa; w[3 + i] = wb; }
        return 6;
    }
    /* 7-point degree-5 rule */
    double s15 = sqrt(15.0);
    double a1 = (6 - s15) / 21, w1 = (155 - s15) / 1200;
    double a2 = (6 + s15) / 21, w2 = (155 + s15) / 1200;
    double P[21] = {1. / 3, 1. / 3, 1. / 3,
                    a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, 1 - 2 * a1, a1, a1,
                    a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, 1 - 2 * a2, a2, a2};
    memcpy(bary, P, sizeof P);
    w[0] = 9.0 / 40.0;
    for (int i = 0; i < 3; i++) { w[1 + i] = w1; w[4 + i] = w2; }
    return 7;
}

static void bary_point(const Tri* t, const double* b, double* x) {
    for (int d = 0; d < 3; d++) x[d] = b[0] * t->p[0][d] + b[1] * t->p[1][d] + b[2] * t->p[2][d];
}

/* Distance from x to the (closed) triangle. */
static double point_tri_dist(const double* x, const Tri* t) {
    double d = 0.0, v[3];
    sub3(x, t->p[0], v);
    d = dot3(v, t->n);
    double p[3] = {x[0] - d * t->n[0], x[1] - d * t->n[1], x[2] - d * t->n[2]};
    int inside = 1;
    for (int i = 0; i < 3; i++) {
        double e[3], q[3], c[3];
        sub3(t->p[(i + 1) % 3], t->p[i], e);
        sub3(p, t->p[i], q);
        cross3(e, q, c);
        if (dot3(c, t->n) < 0) inside = 0;
    }
    if (inside) return fabs(d);
    double best = 1e300;
    for (int i = 0; i < 3; i++) {
        const double* a = t->p[i];
        const double* b = t->p[(i + 1) % 3];
        double ab[3], ax[3];
        sub3(b, a, ab);
        sub3(x, a, ax);
        double s = dot3(ax, ab) / dot3(ab, ab);
        if (s < 0) s = 0;
        if (s > 1) s = 1;
        double q[3] = {a[0] + s * ab[0] - x[0], a[1] + s * ab[1] - x[1], a[2] + s * ab[2] - x[2]};
        double dd = norm3(q);
        if (dd < best) best = dd;
    }
    return best;
}

static double point_tri_maxdist(const double* x, const Tri* t) {
    double best = 0;
    for (int i = 0; i < 3; i++) {
        double v[3];
        sub3(t->p[i], x, v);
        double dd = norm3(v);
        if (dd > best) best = dd;
    }
    return best;
}

/* ------------------------------------------------------------ polar nodes */
typedef struct {
    double y[3];
    double R;
    double w;
} Node;

typedef struct {
    int nt, nr;
    double gt_x[16], gt_w[16], gr_x[16], gr_w[16];
} Rule1D;

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/*
 * Nodes and weights for int_T F(y) dA(y), F smooth except for the point x
 * (1/R-type singularities) and the spheres |x - y| = j * shell (shell > 0).
 * Returns the node count (<= cap).
 */
static int polar_nodes(const double* x, const Tri* T, double shell, const Rule1D* r1, Node* out, int cap) {
    double v0[3];
    sub3(x, T->p[0], v0);
    double d = dot3(v0, T->n);
    double ad = fabs(d);
    double p[3] = {x[0] - d * T->n[0], x[1] - d * T->n[1], x[2] - d * T->n[2]};
    const double tiny = 1e-10 * T->diam;
    int use_sinh = ad > tiny;
    int cnt = 0;
    for (int ei = 0; ei < 3; ei++) {
        const double* a = T->p[ei];
        const double* b = T->p[(ei + 1) % 3];
        double va[3], vb[3], cr[3];
        sub3(a, p, va);
        sub3(b, p, vb);
        cross3(va, vb, cr);
        double s2 = dot3(cr, T->n);
        if (fabs(s2) < 1e-13 * T->diam * T->diam) continue;
        double sgn = s2 > 0 ? 1.0 : -1.0;
        double la = norm3(va);
        double e1[3] = {va[0] / la, va[1] / la, va[2] / la};
        double pr = dot3(vb, e1);
        double e2[3] = {vb[0] - pr * e1[0], vb[1] - pr * e1[1], vb[2] - pr * e1[2]};
        double l2 = norm3(e2);
        for (int k = 0; k < 3; k++) e2[k] /= l2;
        double Theta = atan2(dot3(vb, e2), dot3(vb, e1));
        double ab[3], ap[3];
        sub3(b, a, ab);
        double lab = norm3(ab);
        double th_[3] = {ab[0] / lab, ab[1] / lab, ab[2] / lab};
        sub3(p, a, ap);
        double s = dot3(ap, th_);
        double hv[3] = {a[0] + s * th_[0] - p[0], a[1] + s * th_[1] - p[1], a[2] + s * th_[2] - p[2]};
        double h = norm3(hv);
        if (h < 1e-300) continue;
        double nn[3] = {hv[0] / h, hv[1] / h, hv[2] / h};
        double thn = atan2(dot3(nn, e2), dot3(nn, e1));
        /* angular breakpoints where shells cross the far edge */
        double tb[72];
        int ntb = 0;
        tb[ntb++] = 0.0;
        if (shell > 0) {
            double Rfoot = sqrt(d * d + h * h);
            double Ra = sqrt(d * d + la * la), Rb = sqrt(d * d + dot3(vb, vb));
            double Rm = Ra > Rb ? Ra : Rb;
            long j0 = (long)ceil(Rfoot / shell), j1 = (long)floor(Rm / shell);
            for (long j = j0; j <= j1 && ntb < 68; j++) {
                double rs = j * shell;
                if (rs <= ad) continue;
                double rho = sqrt(rs * rs - d * d);
                if (rho <= h) continue;
                double del = acos(h / rho);
                double c1 = thn - del, c2 = thn + del;
                if (c1 > 1e-14 && c1 < Theta - 1e-14) tb[ntb++] = c1;
                if (c2 > 1e-14 && c2 < Theta - 1e-14) tb[ntb++] = c2;
            }
        }
        tb[ntb++] = Theta;
        qsort(tb, ntb, sizeof(double), cmp_double);
        for (int ti = 0; ti + 1 < ntb; ti++) {
            double t0 = tb[ti], t1 = tb[ti + 1];
            if (t1 - t0 < 1e-15) continue;
            for (int gi = 0; gi < r1->nt; gi++) {
                double th = t0 + (t1 - t0) * r1->gt_x[gi];
                double wth = (t1 - t0) * r1->gt_w[gi];
                double ct = cos(th), st = sin(th);
                double u[3] = {ct * e1[0] + st * e2[0], ct * e1[1] + st * e2[1], ct * e1[2] + st * e2[2]};
                double un = dot3(u, nn);
                if (un <= 1e-14) continue;
                double rhoe = h / un;
                double rb[80];
                int nrb = 0;
                double hi;
                if (use_sinh) {
                    hi = asinh(rhoe / ad);
                    rb[nrb++] = 0.0;
                    if (hi > 1.0) rb[nrb++] = 1.0;
                    if (hi > 3.0) rb[nrb++] = 3.0;
                    if (shell > 0) {
                        double Re = sqrt(d * d + rhoe * rhoe);
                        long j0 = (long)floor(ad / shell) + 1, j1 = (long)floor(Re / shell);
                        for (long j = j0; j <= j1 && nrb < 76; j++) {
                            double sj = acosh(j * shell / ad);
                            if (sj > 1e-14 && sj < hi - 1e-14) rb[nrb++] = sj;
                        }
                    }
                } else {
                    hi = rhoe;
                    rb[nrb++] = 0.0;
                    if (shell > 0) {
                        long j1 = (long)floor(rhoe / shell);
                        for (long j = 1; j <= j1 && nrb < 76; j++) {
                            double sj = j * shell;
                            if (sj > 1e-14 && sj < hi - 1e-14) rb[nrb++] = sj;
                        }
                    }
                }
                rb[nrb++] = hi;
                qsort(rb, nrb, sizeof(double), cmp_double);
                for (int ri = 0; ri + 1 < nrb; ri++) {
                    double s0 = rb[ri], s1 = rb[ri + 1];
                    if (s1 - s0 < 1e-15) continue;
                    for (int gj = 0; gj < r1->nr; gj++) {
                        double sv = s0 + (s1 - s0) * r1->gr_x[gj];
                        double ws = (s1 - s0) * r1->gr_w[gj];
                        double rho, R, jac;
                        if (use_sinh) {
                            double sh = sinh(sv), ch = cosh(sv);
                            rho = ad * sh;
                            R = ad * ch;
                            jac = ad * ad * sh * ch;
                        } else {
                            rho = sv;
                            R = sv;
                            jac = sv;
                        }
                        if (cnt >= cap) return cnt;
                        Node* nd = &out[cnt++];
                        for (int k = 0; k < 3; k++) nd->y[k] = p[k] + rho * u[k];
                        nd->R = R;
                        nd->w = sgn * wth * ws * jac;
                    }
                }
            }
        }
    }
    return cnt;
}

/* Plain symmetric rule on T (far interactions). */
static int plain_nodes(const double* x, const Tri* T, int nq, Node* out) {
    double bary[21], w[7];
    int n = tri_rule(nq, bary, w);
    for (int q = 0; q < n; q++) {
        bary_point(T, bary + 3 * q, out[q].y);
        double v[3];
        sub3(x, out[q].y, v);
        out[q].R = norm3(v);
        out[q].w = w[q] * T->area;
    }
    return n;
}

/* ===================================================================== */
/*                 time-domain assembly (one medium)                      */
/* ===================================================================== */

/* kinds stored per medium */
enum { K_AT = 0, K_AK, K_HT, K_HK, K_TT, K_TK, NKIND };
/* moment slots per lag */
enum { M_TA = 0, M_TH = 4, M_HH = 8, M_TT = 9, M_KA = 13, M_KH = 17, M_KTD = 21, M_KTS = 25, NMOM = 29 };

typedef struct {
    int nv, nf, ne;
    const double* V;
    const int* F;
    const int* EV;
    const int* EF;
    const int* EO;
    double c, dt, tmax;
    int kmax, nq, nthreads, far_plain;
    Rule1D r1, r1far;
    Tri* tris;
    int* face_edges;      /* [nf][3] edge ids */
    double* face_sgn;     /* [nf][3] +1 if face is c^+ of the edge */
    int* face_opp;        /* [nf][3] opposite vertex */
    /* output half rows: per (edge, side) */
    struct HalfRow* halves;
    int next_face;
    pthread_mutex_t lock;
} TDCtx;

/* compressed row for one kind: entries (n, k0, cnt, values) */
typedef struct {
    int nent;
    int* col;
    int* k0;
    int* cnt;
    int64_t* voff;
    double* val;
    int64_t nval;
    /* tail (only K~): per entry: first tail lag a (>= k0+cnt) and constant; a = -1 none */
    int* ta;
    double* tc;
} KRow;

typedef struct HalfRow {
    KRow k[NKIND];
} HalfRow;

static void accum_mom(double* m, double v, const double* y) {
    m[0] += v;
    m[1] += v * y[0];
    m[2] += v * y[1];
    m[3] += v * y[2];
}

/*
 * Temporal factors of one retarded interaction with R / (c dt) = j + phi,
 * 0 <= phi < 1 (paper Section V-A): p_0 is the unit pulse on (-dt, 0), h_0 the
 * hat of half-width dt, and q_0 the average of h_0 over one step, q_0(s) =
 * (1/dt) int_{s-dt}^{s} h_0 (the compatibility Eq. (hq)). The lag-k factor of
 * a basis b is b(k dt - R/c), so lag j + i takes b((i - phi) dt):
 *   w[0..1]   = dt   h_0'  at lags j, j+1
 *   w[2..4]   = dt^2 q_0'' at lags j .. j+2
 *   w[5..7]   =      q_0   at lags j .. j+2
 *   w[8]      =      p_0   at lag j
 *   w[9..10]  =      h_0   at lags j, j+1
 *   w[11..13] = dt   q_0'  at lags j .. j+2
 *   w[14..15] = (1/dt) int_{-inf}^{s} p_0, the ramp of the K~ constant tail, at lags j, j+1
 * (the time derivative of the ramp is p_0, w[8] at lag j and 0 after).
 */
void asm_time_weights(double phi, double* w) {
    const double om = 1.0 - phi;
    w[0] = 1.0;
    w[1] = -1.0;
    w[2] = 1.0;
    w[3] = -2.0;
    w[4] = 1.0;
    w[5] = 0.5 * om * om;
    w[6] = 0.5 - om * om + om;
    w[7] = 0.5 * phi * phi;
    w[8] = 1.0;
    w[9] = om;
    w[10] = phi;
    w[11] = om;
    w[12] = 2.0 * phi - 1.0;
    w[13] = -phi;
    w[14] = om;
    w[15] = 1.0;
}

/*
 * Accumulate, for one outer point x and source triangle, the lag moments
 * mom[(k - kbase) * NMOM + slot]. Returns nothing; caller sizes the window.
 */
static void td_node(const TDCtx* C, const Node* nd, int kbase, int W, double* mom, unsigned char* hit) {
    double R = nd->R;
    if (R <= 0) return;
    double c = C->c, dt = C->dt;
    double s = R / (c * dt);
    int j = (int)floor(s);
    double phi = s - j;
    int l = j - kbase;
    if (l < 0 || l + 2 >= W) return; /* cannot happen with a correct window */
    hit[l] |= 1 | 2 | 4;
    hit[l + 1] |= 1 | 2 | 8;
    hit[l + 2] |= 2;
    double iR = 1.0 / R, iR2 = iR * iR, iR3 = iR2 * iR;
    double w = nd->w;
    double* a0 = mom + (size_t)l * NMOM;
    double* a1 = a0 + NMOM;
    double* a2 = a1 + NMOM;
    const double* y = nd->y;
    double wr = w * iR, idt = 1.0 / dt, idt2 = idt * idt;
    double tw[16];
    asm_time_weights(phi, tw);
    /* A: h_0' at lags j, j+1 */
    accum_mom(a0 + M_TA, wr * tw[0] * idt, y);
    accum_mom(a1 + M_TA, wr * tw[1] * idt, y);
    /* Ah singular: q_0'' at lags j .. j+2 */
    accum_mom(a0 + M_TH, wr * tw[2] * idt2, y);
    accum_mom(a1 + M_TH, wr * tw[3] * idt2, y);
    accum_mom(a2 + M_TH, wr * tw[4] * idt2, y);
    /* Ah hypersingular: q_0 values */
    a0[M_HH] += wr * tw[5];
    a1[M_HH] += wr * tw[6];
    a2[M_HH] += wr * tw[7];
    /* At: p_0 at lag j */
    accum_mom(a0 + M_TT, wr * tw[8], y);
    /* K kernels: psi = chi'/(c R^2) + chi/R^3 */
    double wk2 = w * iR2 / c, wk3 = w * iR3;
    /* K with h_0 (A), q_0 (Ah) and the ramp of the K~ tail: chi' / (c R^2) + chi / R^3 */
    accum_mom(a0 + M_KA, wk2 * tw[0] * idt + wk3 * tw[9], y);
    accum_mom(a1 + M_KA, wk2 * tw[1] * idt + wk3 * tw[10], y);
    accum_mom(a0 + M_KH, wk2 * tw[2] * idt2 + wk3 * tw[11] * idt, y);
    accum_mom(a1 + M_KH, wk2 * tw[3] * idt2 + wk3 * tw[12] * idt, y);
    accum_mom(a2 + M_KH, wk2 * tw[4] * idt2 + wk3 * tw[13] * idt, y);
    accum_mom(a0 + M_KTD, wk2 * tw[8] + wk3 * tw[14] * dt, y);
    accum_mom(a1 + M_KTS, wk3 * tw[15] * dt, y);
}

typedef struct {
    TDCtx* C;
    /* per thread scratch */
    double* buf;       /* [3 local edges][NKIND+1][L][ne]: kind index NKIND = K~ step */
    int* kmin;         /* [3][NKIND+1][ne] */
    int* kmax;
    int L;
    Node* nodes;
    int cap;
    double* mom;
    int momcap;
} TDThread;

#define SLOT(th, le, kind, k, n) ((th)->buf[((((size_t)(le) * (NKIND + 1) + (kind)) * (th)->L + (k)) * (size_t)(th)->C->ne) + (n)])

static void touch(TDThread* th, int le, int kind, int k, int n) {
    size_t i = ((size_t)le * (NKIND + 1) + kind) * th->C->ne + n;
    if (k < th->kmin[i]) th->kmin[i] = k;
    if (k > th->kmax[i]) th->kmax[i] = k;
}

static void finalize_half(TDThread* th, int le, HalfRow* hr) {
    TDCtx* C = th->C;
    int ne = C->ne;
    for (int kind = 0; kind < NKIND; kind++) {
        KRow* kr = &hr->k[kind];
        /* count */
        int nent = 0;
        int64_t nval = 0;
        int kcap = (kind == K_AT || kind == K_AK) ? C->kmax : (kind == K_HT || kind == K_HK) ? C->kmax + 1 : C->kmax - 1;
        for (int n = 0; n < ne; n++) {
            size_t i = ((size_t)le * (NKIND + 1) + kind) * ne + n;
            int lo = th->kmin[i], hi = th->kmax[i];
            if (kind == K_TK) {
                size_t is = ((size_t)le * (NKIND + 1) + NKIND) * ne + n;
                if (th->kmin[is] < lo) lo = th->kmin[is];
                if (th->kmax[is] > hi) hi = th->kmax[is];
                /* explicit window ends one lag before the constant tail starts */
                if (hi > kcap) hi = kcap;
            } else if (hi > kcap) hi = kcap;
            if (lo > hi) continue;
            nent++;
            nval += hi - lo + 1;
        }
        kr->nent = nent;
        kr->nval = nval;
        kr->col = (int*)malloc(sizeof(int) * (nent ? nent : 1));
        kr->k0 = (int*)malloc(sizeof(int) * (nent ? nent : 1));
        kr->cnt = (int*)malloc(sizeof(int) * (nent ? nent : 1));
        kr->voff = (int64_t*)malloc(sizeof(int64_t) * (nent ? nent : 1));
        kr->val = (double*)malloc(sizeof(double) * (nval ? nval : 1));
        kr->ta = NULL;
        kr->tc = NULL;
        if (kind == K_TK) {
            kr->ta = (int*)malloc(sizeof(int) * (nent ? nent : 1));
            kr->tc = (double*)malloc(sizeof(double) * (nent ? nent : 1));
        }
        int e = 0;
        int64_t vo = 0;
        for (int n = 0; n < ne; n++) {
            size_t i = ((size_t)le * (NKIND + 1) + kind) * ne + n;
            int lo = th->kmin[i], hi = th->kmax[i];
            int slo = 1 << 30, shi = -1;
            if (kind == K_TK) {
                size_t is = ((size_t)le * (NKIND + 1) + NKIND) * ne + n;
                slo = th->kmin[is];
                shi = th->kmax[is];
                if (slo < lo) lo = slo;
                if (shi > hi) hi = shi;
            }
            int full_hi = hi;
            if (hi > kcap) hi = kcap;
            if (lo > hi) {
                /* still clear the scratch */
                for (int k = th->kmin[i]; k <= th->kmax[i]; k++) SLOT(th, le, kind, k, n) = 0.0;
                if (kind == K_TK)
                    for (int k = slo; k <= shi; k++) SLOT(th, le, NKIND, k, n) = 0.0;
                th->kmin[i] = 1 << 30;
                th->kmax[i] = -1;
                if (kind == K_TK) {
                    size_t is = ((size_t)le * (NKIND + 1) + NKIND) * ne + n;
                    th->kmin[is] = 1 << 30;
                    th->kmax[is] = -1;
                }
                continue;
            }
            kr->col[e] = n;
            kr->k0[e] = lo;
            kr->cnt[e] = hi - lo + 1;
            kr->voff[e] = vo;
            double run = 0.0;
            for (int k = lo; k <= full_hi; k++) {
                double v = SLOT(th, le, kind, k, n);
                if (kind == K_TK) {
                    run += SLOT(th, le, NKIND, k, n);
                    v += run;
                }
                if (k <= hi) kr->val[vo + (k - lo)] = v;
            }
            if (kind == K_TK) {
                /* tail: constant `run` from lag full_hi + 1 on (all nodes arrived) */
                int a = full_hi + 1;
                kr->ta[e] = a;
                kr->tc[e] = run;
            }
            vo += hi - lo + 1;
            e++;
            for (int k = th->kmin[i]; k <= th->kmax[i]; k++) SLOT(th, le, kind, k, n) = 0.0;
            th->kmin[i] = 1 << 30;
            th->kmax[i] = -1;
            if (kind == K_TK) {
                size_t is = ((size_t)le * (NKIND + 1) + NKIND) * ne + n;
                for (int k = th->kmin[is]; k <= th->kmax[is]; k++) SLOT(th, le, NKIND, k, n) = 0.0;
                th->kmin[is] = 1 << 30;
                th->kmax[is] = -1;
            }
        }
    }
}

static void* td_worker(void* arg) {
    TDThread* th = (TDThread*)arg;
    TDCtx* C = th->C;
    int ne = C->ne;
    double bary[21], wq[7];
    int nq = tri_rule(C->nq, bary, wq);
    double cdt = C->c * C->dt;
    const double i4pi = 1.0 / (4.0 * PI);
    for (;;) {
        pthread_mutex_lock(&C->lock);
        int S = C->next_face++;
        pthread_mutex_unlock(&C->lock);
        if (S >= C->nf) break;
        const Tri* TS = &C->tris[S];
        for (int q = 0; q < nq; q++) {
            double x[3];
            bary_point(TS, bary + 3 * q, x);
            double wx = wq[q] * TS->area;
            /* test functions at x */
            double fm[3][3], divm[3];
            for (int le = 0; le < 3; le++) {
                int o = C->face_opp[3 * S + le];
                double sg = C->face_sgn[3 * S + le];
                for (int d = 0; d < 3; d++) fm[le][d] = sg * (x[d] - C->V[3 * o + d]) / (2.0 * TS->area);
                divm[le] = sg / TS->area;
            }
            for (int Rf = 0; Rf < C->nf; Rf++) {
                const Tri* TR = &C->tris[Rf];
                double rmin = (Rf == S) ? 0.0 : point_tri_dist(x, TR);
                double rmax = point_tri_maxdist(x, TR);
                int jlo = (int)floor(rmin / cdt), jhi = (int)floor(rmax / cdt);
                int W = jhi - jlo + 4;
                if (W * NMOM > th->momcap) {
                    th->momcap = W * NMOM * 2;
                    th->mom = (double*)realloc(th->mom, sizeof(double) * th->momcap);
                }
                memset(th->mom, 0, sizeof(double) * W * NMOM);
                int nn;
                double cdist[3];
                sub3(x, TR->cen, cdist);
                double dc = norm3(cdist);
                int coplanar = (Rf == S);
                if (!coplanar) {
                    double v0[3];
                    sub3(x, TR->p[0], v0);
                    if (fabs(dot3(v0, TR->n)) < 1e-10 * TR->diam && fabs(dot3(TS->n, TR->n)) > 1.0 - 1e-12) coplanar = 1;
                }
                if ((jlo == jhi || C->far_plain) && dc > 3.0 * TR->diam)
                    nn = plain_nodes(x, TR, C->far_plain ? C->far_plain : 7, th->nodes);
                else if (dc > 3.0 * TR->diam)
                    nn = polar_nodes(x, TR, cdt, &C->r1far, th->nodes, th->cap);
                else
                    nn = polar_nodes(x, TR, cdt, &C->r1, th->nodes, th->cap);
                unsigned char hit[4096];
                if (W > 4096) W = 4096;
                memset(hit, 0, (size_t)W);
                for (int i = 0; i < nn; i++) td_node(C, &th->nodes[i], jlo, W, th->mom, hit);
                /* contract with test and source RWGs */
                for (int jn = 0; jn < 3; jn++) {
                    int n = C->face_edges[3 * Rf + jn];
                    double sn = C->face_sgn[3 * Rf + jn];
                    const double* on = &C->V[3 * C->face_opp[3 * Rf + jn]];
                    double cn = sn / (2.0 * TR->area);
                    double divn = sn / TR->area;
                    for (int l = 0; l < W; l++) {
                        int k = jlo + l;
                        const double* M = th->mom + (size_t)l * NMOM;
                        if (!hit[l]) continue;
                        double MT[4][3];
                        const int tslots[3] = {M_TA, M_TH, M_TT};
                        for (int ts = 0; ts < 3; ts++)
                            for (int d = 0; d < 3; d++)
                                MT[ts][d] = cn * (M[tslots[ts] + 1 + d] - on[d] * M[tslots[ts]]);
                        double MK[4][3];
                        const int kslots[4] = {M_KA, M_KH, M_KTD, M_KTS};
                        for (int ks = 0; ks < 4; ks++) {
                            const double* kk = M + kslots[ks];
                            double t1[3] = {kk[1] - kk[0] * on[0], kk[2] - kk[0] * on[1], kk[3] - kk[0] * on[2]};
                            double c1[3], c2[3];
                            cross3(t1, x, c1);
                            cross3(on, kk + 1, c2);
                            for (int d = 0; d < 3; d++) MK[ks][d] = cn * (c1[d] + c2[d]);
                        }
                        for (int le = 0; le < 3; le++) {
                            double ft = -wx * i4pi / C->c;
                            double vAT = ft * dot3(fm[le], MT[0]);
                            double vHT = ft * C->tmax * dot3(fm[le], MT[1]) -
                                         wx * C->c * C->tmax * i4pi * divm[le] * divn * M[M_HH];
                            double vTT = ft / C->tmax * dot3(fm[le], MT[2]);
                            double vAK = 0, vHK = 0, vTKd = 0, vTKs = 0;
                            if (!coplanar) {
                                double fk = wx * i4pi;
                                vAK = fk * dot3(fm[le], MK[0]);
                                vHK = fk * C->tmax * dot3(fm[le], MK[1]);
                                vTKd = fk / C->tmax * dot3(fm[le], MK[2]);
                                vTKs = fk / C->tmax * dot3(fm[le], MK[3]);
                            }
                            if (k < th->L) {
                                unsigned char hb = hit[l];
                                if (hb & 1) {
                                    SLOT(th, le, K_AT, k, n) += vAT; touch(th, le, K_AT, k, n);
                                    SLOT(th, le, K_AK, k, n) += vAK; touch(th, le, K_AK, k, n);
                                }
                                if (hb & 2) {
                                    SLOT(th, le, K_HT, k, n) += vHT; touch(th, le, K_HT, k, n);
                                    SLOT(th, le, K_HK, k, n) += vHK; touch(th, le, K_HK, k, n);
                                }
                                if (hb & 4) {
                                    SLOT(th, le, K_TT, k, n) += vTT; touch(th, le, K_TT, k, n);
                                    SLOT(th, le, K_TK, k, n) += vTKd; touch(th, le, K_TK, k, n);
                                }
                                if (hb & 8) {
                                    SLOT(th, le, NKIND, k, n) += vTKs; touch(th, le, NKIND, k, n);
                                }
                            }
                        }
                    }
                }
            }
        }
        /* emit the three half rows of this face */
        for (int le = 0; le < 3; le++) {
            int m = C->face_edges[3 * S + le];
            int side = C->face_sgn[3 * S + le] > 0 ? 0 : 1;
            finalize_half(th, le, &C->halves[2 * m + side]);
        }
    }
    (void)ne;
    return NULL;
}

/* Result handle */
typedef struct {
    int ne, kmax;
    /* merged rows, per kind: CSR-like */
    int64_t* rowptr[NKIND];
    int* col[NKIND];
    int* k0[NKIND];
    int* cnt[NKIND];
    int64_t* voff[NKIND];
    double* val[NKIND];
    int64_t nent[NKIND], nval[NKIND];
    int* ta;  /* tail for K~ per entry */
    double* tc;
} TDResult;

static void free_krow(KRow* k) {
    free(k->col);
    free(k->k0);
    free(k->cnt);
    free(k->voff);
    free(k->val);
    free(k->ta);
    free(k->tc);
}

/*
 * Merge the two halves (from c^+_m and c^-_m) of every row. A half h of an
 * entry holds an explicit window [a_h, b_h] and, for K~, a constant tail C_h
 * from lag t_h = b_h + 1 on (t_h > kmax - 1 means no tail inside the kept
 * lags). The merged entry keeps explicit values on [min a_h, T - 1] with
 * T = max t_h over the present halves (clipped to the kept lags) and the tail
 * sum C = sum C_h from T on.
 */
typedef struct {
    int lo, hi, tail;
} MWin;

static MWin merged_window(int kind, int kcap, KRow* const* hs, const int* ix, int nh) {
    MWin w = {1 << 30, -1, 1 << 30};
    for (int h = 0; h < nh; h++) {
        int a = hs[h]->k0[ix[h]], b = a + hs[h]->cnt[ix[h]] - 1;
        if (a < w.lo) w.lo = a;
        if (b > w.hi) w.hi = b;
    }
    if (kind == K_TK) {
        int T = -1;
        for (int h = 0; h < nh; h++) {
            int t = hs[h]->ta[ix[h]];
            if (t > T) T = t;
        }
        if (T - 1 > w.hi) w.hi = T - 1;
        if (w.hi > kcap) w.hi = kcap;
        w.tail = w.hi + 1;
    }
    return w;
}

static void merge_rows(TDCtx* C, TDResult* res) {
    int ne = C->ne;
    for (int kind = 0; kind < NKIND; kind++) {
        int kcap = (kind == K_AT || kind == K_AK) ? C->kmax : (kind == K_HT || kind == K_HK) ? C->kmax + 1 : C->kmax - 1;
        int64_t* rp = (int64_t*)calloc(ne + 1, sizeof(int64_t));
        int64_t tot = 0;
        for (int pass = 0; pass < 2; pass++) {
            int64_t vo = 0;
            for (int m = 0; m < ne; m++) {
                KRow* h0 = &C->halves[2 * m].k[kind];
                KRow* h1 = &C->halves[2 * m + 1].k[kind];
                int i = 0, j = 0, ent = 0;
                int64_t e = pass ? rp[m] : 0;
                while (i < h0->nent || j < h1->nent) {
                    int n0 = i < h0->nent ? h0->col[i] : 1 << 30;
                    int n1 = j < h1->nent ? h1->col[j] : 1 << 30;
                    KRow* hs[2];
                    int ix[2], nh = 0;
                    if (n0 <= n1) { hs[nh] = h0; ix[nh++] = i++; }
                    if (n1 <= n0) { hs[nh] = h1; ix[nh++] = j++; }
                    MWin w = merged_window(kind, kcap, hs, ix, nh);
                    int len = w.hi - w.lo + 1;
                    if (pass == 1) {
                        res->col[kind][e] = hs[0]->col[ix[0]];
                        res->k0[kind][e] = w.lo;
                        res->cnt[kind][e] = len;
                        res->voff[kind][e] = vo;
                        double* dst = res->val[kind] + vo;
                        double tail = 0.0;
                        for (int h = 0; h < nh; h++) {
                            int a = hs[h]->k0[ix[h]], cn = hs[h]->cnt[ix[h]];
                            const double* src = hs[h]->val + hs[h]->voff[ix[h]];
                            for (int q = 0; q < cn; q++) dst[a - w.lo + q] += src[q];
                            if (kind == K_TK) {
                                int t = hs[h]->ta[ix[h]];
                                double cst = hs[h]->tc[ix[h]];
                                for (int k = t; k <= w.hi; k++) dst[k - w.lo] += cst;
                                tail += cst;
                            }
                        }
                        if (kind == K_TK) {
                            res->ta[e] = w.tail;
                            res->tc[e] = tail;
                        }
                        e++;
                    }
                    vo += len;
                    ent++;
                }
                if (pass == 0) rp[m + 1] = ent;
            }
            if (pass == 0) {
                for (int m = 0; m < ne; m++) rp[m + 1] += rp[m];
                tot = vo;
                int64_t nent = rp[ne];
                res->rowptr[kind] = rp;
                res->nent[kind] = nent;
                res->nval[kind] = tot;
                res->col[kind] = (int*)malloc(sizeof(int) * (nent ? nent : 1));
                res->k0[kind] = (int*)malloc(sizeof(int) * (nent ? nent : 1));
                res->cnt[kind] = (int*)malloc(sizeof(int) * (nent ? nent : 1));
                res->voff[kind] = (int64_t*)malloc(sizeof(int64_t) * (nent ? nent : 1));
                res->val[kind] = (double*)calloc(tot ? tot : 1, sizeof(double));
                if (kind == K_TK) {
                    res->ta = (int*)malloc(sizeof(int) * (nent ? nent : 1));
                    res->tc = (double*)malloc(sizeof(double) * (nent ? nent : 1));
                }
            }
        }
    }
}

void* asm_td_run(int nv, const double* V, int nf, const int* F, int ne, const int* EV, const int* EF,
                 const int* EO, double c, double dt, double tmax, int kmax, int nq, int ntheta, int nrad,
                 int nthreads, int far_plain) {
    TDCtx C;
    memset(&C, 0, sizeof C);
    C.nv = nv;
    C.nf = nf;
    C.ne = ne;
    C.V = V;
    C.F = F;
    C.EV = EV;
    C.EF = EF;
    C.EO = EO;
    C.c = c;
    C.dt = dt;
    C.tmax = tmax;
    C.kmax = kmax;
    C.nq = nq;
    C.nthreads = nthreads < 1 ? 1 : nthreads;
    C.far_plain = far_plain;
    C.r1.nt = ntheta;
    C.r1.nr = nrad;
    gauss_legendre01(ntheta, C.r1.gt_x, C.r1.gt_w);
    gauss_legendre01(nrad, C.r1.gr_x, C.r1.gr_w);
    C.r1far.nt = ntheta > 2 ? 2 : ntheta;
    C.r1far.nr = nrad > 3 ? 3 : nrad;
    gauss_legendre01(C.r1far.nt, C.r1far.gt_x, C.r1far.gt_w);
    gauss_legendre01(C.r1far.nr, C.r1far.gr_x, C.r1far.gr_w);
    C.tris = (Tri*)malloc(sizeof(Tri) * nf);
    for (int f = 0; f < nf; f++) make_tri(V, F + 3 * f, &C.tris[f]);
    C.face_edges = (int*)malloc(sizeof(int) * 3 * nf);
    C.face_sgn = (double*)malloc(sizeof(double) * 3 * nf);
    C.face_opp = (int*)malloc(sizeof(int) * 3 * nf);
    int* fill = (int*)calloc(nf, sizeof(int));
    for (int e = 0; e < ne; e++) {
        for (int side = 0; side < 2; side++) {
            int f = EF[2 * e + side];
            int s = fill[f]++;
            C.face_edges[3 * f + s] = e;
            C.face_sgn[3 * f + s] = side == 0 ? 1.0 : -1.0;
            C.face_opp[3 * f + s] = EO[2 * e + side];
        }
    }
    free(fill);
    C.halves = (HalfRow*)calloc((size_t)2 * ne, sizeof(HalfRow));
    C.next_face = 0;
    pthread_mutex_init(&C.lock, NULL);
    int L = kmax + 4;
    TDThread* th = (TDThread*)calloc(C.nthreads, sizeof(TDThread));
    pthread_t* tid = (pthread_t*)malloc(sizeof(pthread_t) * C.nthreads);
    for (int t = 0; t < C.nthreads; t++) {
        th[t].C = &C;
        th[t].L = L;
        th[t].buf = (double*)calloc((size_t)3 * (NKIND + 1) * L * ne, sizeof(double));
        th[t].kmin = (int*)malloc(sizeof(int) * 3 * (NKIND + 1) * ne);
        th[t].kmax = (int*)malloc(sizeof(int) * 3 * (NKIND + 1) * ne);
        for (int i = 0; i < 3 * (NKIND + 1) * ne; i++) {
            th[t].kmin[i] = 1 << 30;
            th[t].kmax[i] = -1;
        }
        th[t].cap = 200000;
        th[t].nodes = (Node*)malloc(sizeof(Node) * th[t].cap);
        th[t].momcap = 64 * NMOM;
        th[t].mom = (double*)malloc(sizeof(double) * th[t].momcap);
        pthread_create(&tid[t], NULL, td_worker, &th[t]);
    }
    for (int t = 0; t < C.nthreads; t++) {
        pthread_join(tid[t], NULL);
        free(th[t].buf);
        free(th[t].kmin);
        free(th[t].kmax);
        free(th[t].nodes);
        free(th[t].mom);
    }
    free(th);
    free(tid);
    TDResult* res = (TDResult*)calloc(1, sizeof(TDResult));
    res->ne = ne;
    res->kmax = kmax;
    merge_rows(&C, res);
    for (int i = 0; i < 2 * ne; i++)
        for (int k = 0; k < NKIND; k++) free_krow(&C.halves[i].k[k]);
    free(C.halves);
    free(C.tris);
    free(C.face_edges);
    free(C.face_sgn);
    free(C.face_opp);
    pthread_mutex_destroy(&C.lock);
    return res;
}

void asm_td_sizes(void* h, int kind, int64_t* nent, int64_t* nval) {
    TDResult* r = (TDResult*)h;
    *nent = r->nent[kind];
    *nval = r->nval[kind];
}

void asm_td_copy(void* h, int kind, int64_t* rowptr, int* col, int* k0, int* cnt, int64_t* voff, double* val,
                 int* ta, double* tc) {
    TDResult* r = (TDResult*)h;
    memcpy(rowptr, r->rowptr[kind], sizeof(int64_t) * (r->ne + 1));
    memcpy(col, r->col[kind], sizeof(int) * r->nent[kind]);
    memcpy(k0, r->k0[kind], sizeof(int) * r->nent[kind]);
    memcpy(cnt, r->cnt[kind], sizeof(int) * r->nent[kind]);
    memcpy(voff, r->voff[kind], sizeof(int64_t) * r->nent[kind]);
    memcpy(val, r->val[kind], sizeof(double) * r->nval[kind]);
    if (kind == K_TK && ta) {
        memcpy(ta, r->ta, sizeof(int) * r->nent[kind]);
        memcpy(tc, r->tc, sizeof(double) * r->nent[kind]);
    }
}

void asm_td_free(void* h) {
    TDResult* r = (TDResult*)h;
    for (int k = 0; k < NKIND; k++) {
        free(r->rowptr[k]);
        free(r->col[k]);
        free(r->k0[k]);
        free(r->cnt[k]);
        free(r->voff[k]);
        free(r->val[k]);
    }
    free(r->ta);
    free(r->tc);
    free(r);
}

/* ===================================================================== */
/*           static operators on the barycentric refinement               */
/* ===================================================================== */
/*
 * T_0^s = (1/D) <<g_m . g_n / (4 pi R)>> and the dual-cell single layer
 * S_vw = (D/(4 pi)) <<phi_v phi_w / R>>, phi_v = 1/(2 d_v A_t) on the refined
 * triangles t of D(v), so that T_0^h = Lambda S Lambda^T.
 * g_n|_t(x) = alpha x + beta; needs the moments I0, Ix, Iy, Ixy of 1/R over
 * refined triangle pairs.
 * kappa > 0: the EFIO with the imaginary wavenumber -i kappa in place of the
 * static one (Section IV-A remark): the kernel 1/R becomes exp(-kappa R)/R
 * (same normalisations 1/D and D); kappa = 0 is the static operator exactly.
 */
typedef struct {
    int nref, ne, nv;
    Tri* rt;
    const int* rvert;     /* dual cell of each refined triangle */
    const int* deg;       /* degree of each primal vertex */
    /* BC entries grouped by refined triangle (CSR) */
    const int64_t* bptr;
    const int* bn;
    const double* ba;
    const double* bb;
    /* dual cell lists */
    const int64_t* cptr;
    const int* ctri;
    const int* v_edges_ptr_dummy;
    double D;
    double kappa;   /* Yukawa decay of the kernel (0: static) */
    int nq;
    Rule1D r1;
    double* half;   /* [2][ne][ne] halves of T_0^s rows */
    const int* ev;  /* edge endpoints: to choose the half */
    double* S;      /* [nv][nv] */
    int next;
    pthread_mutex_t lock;
} STCtx;

static void static_moments(const STCtx* C, const Tri* A, const Tri* B, int same, Node* nodes, int cap,
                           double* I0, double* Ix, double* Iy, double* Ixy) {
    double bary[21], w[7];
    double dist[3];
    sub3(A->cen, B->cen, dist);
    double dc = norm3(dist);
    double sz = A->diam > B->diam ? A->diam : B->diam;
    int nqo = C->nq;
    if (!same && dc > 8 * sz) nqo = 1;
    else if (!same && dc > 4 * sz) nqo = 3;
    int n = tri_rule(nqo, bary, w);
    *I0 = 0;
    Ix[0] = Ix[1] = Ix[2] = 0;
    Iy[0] = Iy[1] = Iy[2] = 0;
    *Ixy = 0;
    for (int q = 0; q < n; q++) {
        double x[3];
        bary_point(A, bary + 3 * q, x);
        double wx = w[q] * A->area;
        int nn;
        if (same || dc <= 4 * sz)
            nn = polar_nodes(x, B, 0.0, &C->r1, nodes, cap);
        else
            nn = plain_nodes(x, B, nqo, nodes);
        double s0 = 0, s1[3] = {0, 0, 0};
        for (int i = 0; i < nn; i++) {
            double v = nodes[i].w / nodes[i].R;
            if (C->kappa > 0.0) v *= exp(-C->kappa * nodes[i].R);
            s0 += v;
            s1[0] += v * nodes[i].y[0];
            s1[1] += v * nodes[i].y[1];
            s1[2] += v * nodes[i].y[2];
        }
        *I0 += wx * s0;
        for (int d = 0; d < 3; d++) {
            Ix[d] += wx * s0 * x[d];
            Iy[d] += wx * s1[d];
        }
        *Ixy += wx * dot3(x, s1);
    }
}

static void* st_worker(void* arg) {
    STCtx* C = (STCtx*)arg;
    int ne = C->ne;
    Node* nodes = (Node*)malloc(sizeof(Node) * 20000);
    double* a_n = (double*)malloc(sizeof(double) * ne);
    double* b_n = (double*)malloc(sizeof(double) * 3 * ne);
    double* Srow = (double*)malloc(sizeof(double) * C->nv);
    for (;;) {
        pthread_mutex_lock(&C->lock);
        int v = C->next++;
        pthread_mutex_unlock(&C->lock);
        if (v >= C->nv) break;
        memset(Srow, 0, sizeof(double) * C->nv);
        for (int64_t ti = C->cptr[v]; ti < C->cptr[v + 1]; ti++) {
            int t = C->ctri[ti];
            const Tri* A = &C->rt[t];
            memset(a_n, 0, sizeof(double) * ne);
            memset(b_n, 0, sizeof(double) * 3 * ne);
            double phit = 1.0 / (2.0 * C->deg[v] * A->area);
            for (int t2 = 0; t2 < C->nref; t2++) {
                const Tri* B = &C->rt[t2];
                double I0, Ix[3], Iy[3], Ixy;
                static_moments(C, A, B, t2 == t, nodes, 20000, &I0, Ix, Iy, &Ixy);
                int w2 = C->rvert[t2];
                Srow[w2] += phit * I0 / (2.0 * C->deg[w2] * B->area);
                for (int64_t b = C->bptr[t2]; b < C->bptr[t2 + 1]; b++) {
                    int n = C->bn[b];
                    double al = C->ba[b];
                    const double* be = C->bb + 3 * b;
                    a_n[n] += al * Ixy + dot3(be, Ix);
                    for (int d = 0; d < 3; d++) b_n[3 * n + d] += al * Iy[d] + be[d] * I0;
                }
            }
            for (int64_t b = C->bptr[t]; b < C->bptr[t + 1]; b++) {
                int m = C->bn[b];
                double al = C->ba[b];
                const double* be = C->bb + 3 * b;
                int side = (C->ev[2 * m] == v) ? 0 : 1;
                double* row = C->half + ((size_t)side * ne + m) * ne;
                for (int n = 0; n < ne; n++)
                    row[n] += (al * a_n[n] + dot3(be, b_n + 3 * n)) / (4.0 * PI * C->D);
            }
        }
        for (int w2 = 0; w2 < C->nv; w2++) C->S[(size_t)v * C->nv + w2] = Srow[w2] * C->D / (4.0 * PI);
    }
    free(nodes);
    free(a_n);
    free(b_n);
    free(Srow);
    return NULL;
}

/*
 * ref_pts: (nref, 3, 3); rvert: dual cell per refined triangle; deg: (nv);
 * bptr/bn/ba/bb: BC entries grouped by refined triangle; cptr/ctri: refined
 * triangles per dual cell; ev: (ne, 2).
 * kappa: decay of the kernel exp(-kappa R)/R (0: the static 1/R).
 * Outputs T0s (ne x ne, row-major) and S (nv x nv).
 */
int asm_static(int nref, const double* ref_pts, const int* rvert, int nv, const int* deg, int ne, const int* ev,
               const int64_t* bptr, const int* bn, const double* ba, const double* bb, const int64_t* cptr,
               const int* ctri, double D, double kappa, int nq, int ntheta, int nrad, int nthreads, double* T0s,
               double* S) {
    STCtx C;
    memset(&C, 0, sizeof C);
    C.nref = nref;
    C.ne = ne;
    C.nv = nv;
    C.rvert = rvert;
    C.deg = deg;
    C.bptr = bptr;
    C.bn = bn;
    C.ba = ba;
    C.bb = bb;
    C.cptr = cptr;
    C.ctri = ctri;
    C.ev = ev;
    C.D = D;
    C.kappa = kappa;
    C.nq = nq;
    C.r1.nt = ntheta;
    C.r1.nr = nrad;
    gauss_legendre01(ntheta, C.r1.gt_x, C.r1.gt_w);
    gauss_legendre01(nrad, C.r1.gr_x, C.r1.gr_w);
    C.rt = (Tri*)malloc(sizeof(Tri) * nref);
    for (int t = 0; t < nref; t++) {
        int idx[3] = {3 * t, 3 * t + 1, 3 * t + 2};
        make_tri(ref_pts, idx, &C.rt[t]);
    }
    C.half = (double*)calloc((size_t)2 * ne * ne, sizeof(double));
    C.S = S;
    pthread_mutex_init(&C.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t* tid = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; t++) pthread_create(&tid[t], NULL, st_worker, &C);
    for (int t = 0; t < nthreads; t++) pthread_join(tid[t], NULL);
    for (size_t i = 0; i < (size_t)ne * ne; i++) T0s[i] = C.half[i] + C.half[(size_t)ne * ne + i];
    free(C.half);
    free(C.rt);
    free(tid);
    pthread_mutex_destroy(&C.lock);
    return 0;
}
