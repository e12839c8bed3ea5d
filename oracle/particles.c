/*
 * FP64 oracle of one particle step: gather, relativistic push (Boris, or Vay's
 * correction of it), move with rotate-back to the meridian plane, triangle walk,
 * charge-conserving scatter.
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow reference code used to check the GPU library.
 * Shares no code with it.  Compiled with -ffp-contract=off so that x86 and Arm
 * builds round identically.
 *
 * Conventions (mesh arrays are produced by oracle/operators.py):
 *   x = z, y = rho in the meridian plane; triangles counter-clockwise.
 *   local edge k of a triangle joins local nodes (k+1)%3 and (k+2)%3 (opposite node k);
 *   edge orientation runs from the lower to the higher global node index.
 *   grad[t][k] = (d lambda_k / dz, d lambda_k / drho).
 *   momenta u = gamma v in the particle's local (rho, phi, z) frame.
 */
#include <math.h>
#include <stdint.h>

/* The plain build (the oracle the tests use) is single-threaded and these expand to
 * nothing.  Built a second time with -fopenmp, for the timed CPU baseline only, the
 * particle loop runs on all host cores and every accumulation into shared arrays is
 * atomic (the order of the sums then varies between runs). */
#ifdef _OPENMP
#include <omp.h>
#define ORACLE_PARALLEL_FOR _Pragma("omp parallel for schedule(dynamic, 4096)")
#define ORACLE_ATOMIC _Pragma("omp atomic")
#else
#define ORACLE_PARALLEL_FOR
#define ORACLE_ATOMIC
#endif

enum { TAG_INTERIOR = 0, TAG_PEC = 1, TAG_AXIS = 2, TAG_ABSORB = 3 };

typedef struct {
    const int32_t *tri_nodes; /* [N2][3] */
    const int32_t *tri_edges; /* [N2][3] */
    const int32_t *tri_nbr;   /* [N2][3] */
    const int32_t *tri_btag;  /* [N2][3] */
    const double *node_zr;    /* [N0][2] */
    const double *grad;       /* [N2][3][2] */
    const double *area;       /* [N2] */
} omesh;

/* tail a / head b (local indices) of local edge k */
static void edge_ends(const int32_t *nodes3, int k, int *a, int *b)
{
    int i = (k + 1) % 3, j = (k + 2) % 3;
    if (nodes3[i] < nodes3[j]) { *a = i; *b = j; }
    else                       { *a = j; *b = i; }
}

/* Eq. current: the segment from ls to le inside triangle t adds
 * w * int W1_e . dr = w * (ls_a le_b - ls_b le_a) to each of the triangle's edges. */
static void deposit_segment(const omesh *m, int t, const double ls[3], const double le[3],
                            double w, double *J)
{
    const int32_t *n3 = m->tri_nodes + 3 * t;
    for (int k = 0; k < 3; k++) {
        int a, b;
        edge_ends(n3, k, &a, &b);
        ORACLE_ATOMIC J[m->tri_edges[3 * t + k]] += w * (ls[a] * le[b] - ls[b] * le[a]);
    }
}

/* Sec. 3.2 gather: E = sum_e E_e W1_e(lambda) (components z, rho). */
static void gather_E(const omesh *m, int t, const double lam[3], const double *E,
                     double *Ez, double *Er)
{
    const int32_t *n3 = m->tri_nodes + 3 * t;
    const double *g = m->grad + 6 * t;
    double ez = 0.0, er = 0.0;
    for (int k = 0; k < 3; k++) {
        int a, b;
        edge_ends(n3, k, &a, &b);
        double Ee = E[m->tri_edges[3 * t + k]];
        ez += Ee * (lam[a] * g[2 * b + 0] - lam[b] * g[2 * a + 0]);
        er += Ee * (lam[a] * g[2 * b + 1] - lam[b] * g[2 * a + 1]);
    }
    *Ez = ez;
    *Er = er;
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    /* components ordered (rho, phi, z), a right-handed frame */
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Eq. DLE solved with Boris's splitting (Sec. 3.3): half electric kick, rotation about B
 * by the angle of t = h B / gamma(u-), half electric kick.  h = q dt / (2 m). */
static void kick_boris(const double u[3], const double Ef[3], const double Bf[3], double h,
                       double c, double out[3])
{
    double um[3], tv[3], sv[3], c1[3], upr[3];
    for (int i = 0; i < 3; i++) um[i] = u[i] + h * Ef[i];
    double gam = sqrt(1.0 + dot3(um, um) / (c * c));
    for (int i = 0; i < 3; i++) tv[i] = h * Bf[i] / gam;
    double t2 = dot3(tv, tv);
    for (int i = 0; i < 3; i++) sv[i] = 2.0 * tv[i] / (1.0 + t2);
    cross3(um, tv, c1);
    for (int i = 0; i < 3; i++) upr[i] = um[i] + c1[i];
    cross3(upr, sv, c1);
    for (int i = 0; i < 3; i++) out[i] = um[i] + c1[i] + h * Ef[i];
}

/* Eq. DLE with the velocity term read as the mean of v^{n-1/2} and v^{n+1/2} (Vay 2008,
 * the correction the paper cites in Sec. 3.3), solved exactly:
 *   u' = u + 2h E + h v x B,  v = u / gamma(u);  tau = h B;
 *   gamma_new^2 is the positive root of g^4 - sigma g^2 - (tau^2 + (u'.tau / c)^2) = 0,
 *   sigma = gamma(u')^2 - tau^2;  t = tau / gamma_new;
 *   u_new = (u' + (u'.t) t + u' x t) / (1 + t^2). */
static void kick_vay(const double u[3], const double Ef[3], const double Bf[3], double h,
                     double c, double out[3])
{
    double v[3], vxb[3], up[3], tau[3], tv[3], c1[3];
    double gam = sqrt(1.0 + dot3(u, u) / (c * c));
    for (int i = 0; i < 3; i++) v[i] = u[i] / gam;
    cross3(v, Bf, vxb);
    for (int i = 0; i < 3; i++) up[i] = u[i] + 2.0 * h * Ef[i] + h * vxb[i];
    for (int i = 0; i < 3; i++) tau[i] = h * Bf[i];
    double tau2 = dot3(tau, tau);
    double ustar = dot3(up, tau) / c;
    double sigma = 1.0 + dot3(up, up) / (c * c) - tau2;
    double gnew = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))));
    for (int i = 0; i < 3; i++) tv[i] = tau[i] / gnew;
    double ut = dot3(up, tv);
    double s = 1.0 / (1.0 + dot3(tv, tv));
    cross3(up, tv, c1);
    for (int i = 0; i < 3; i++) out[i] = s * (up[i] + ut * tv[i] + c1[i]);
}

static void kick(int pusher, const double u[3], const double Ef[3], const double Bf[3],
                 double h, double c, double out[3])
{
    if (pusher == 1) kick_vay(u, Ef, Bf, h, c, out);
    else kick_boris(u, Ef, Bf, h, c, out);
}

/* The velocity update alone, for n particles with given fields (rows of 3, local
 * (rho, phi, z) components): pins of the two pushers. */
int oracle_kick(int pusher, int64_t n, const double *u, const double *Ef, const double *Bf,
                double h, double c, double *out)
{
    for (int64_t p = 0; p < n; p++) kick(pusher, u + 3 * p, Ef + 3 * p, Bf + 3 * p, h, c, out + 3 * p);
    return 0;
}

/*
 * Push all particles one step.  On entry: tri/lam at step n, u at n-1/2; E at n,
 * Bavg = (B^{n+1/2} + B^{n-1/2}) / 2 per face.  On exit: tri/lam at n+1 (tri = -1 for
 * absorbed particles), u at n+1/2.  J (N1) receives q_src/dt * int W1 . dr, Q (N0)
 * receives q_src * lambda at the new positions, Qabs (N0) the charge of particles
 * absorbed this step at their wall position.  counters: [0] absorbed, [1] walk-cap
 * overflows, [2] edge crossings.
 */
int oracle_push(const int32_t *tri_nodes, const int32_t *tri_edges, const int32_t *tri_nbr,
                const int32_t *tri_btag, const double *node_zr, const double *grad,
                const double *area, const double *E, const double *Bavg, double bz,
                double dt, double qm, double c, double q_src, int max_cross, int pusher,
                int64_t np, int32_t *tri, double *lam, double *u, double *J, double *Q,
                double *Qabs, int64_t *counters)
{
    omesh m = {tri_nodes, tri_edges, tri_nbr, tri_btag, node_zr, grad, area};
    const double h = 0.5 * qm * dt;
    const double wJ = q_src / dt;
    ORACLE_PARALLEL_FOR
    for (int64_t p = 0; p < np; p++) {
        int t = tri[p];
        if (t < 0) continue;
        double l[3] = {lam[3 * p], lam[3 * p + 1], lam[3 * p + 2]};
        const int32_t *n3 = tri_nodes + 3 * t;

        /* gather (Sec. 3.2): E at r^n; B_phi = Bavg W2 = Bavg / A; guide field B_z */
        double Ez, Er;
        gather_E(&m, t, l, E, &Ez, &Er);
        double Ef[3] = {Er, 0.0, Ez};
        double Bf[3] = {0.0, Bavg[t] / area[t], bz};

        /* relativistic push (Eq. DLE) */
        double up[3];
        kick(pusher, u + 3 * p, Ef, Bf, h, c, up);

        /* move (Eq. DNE) in the Cartesian frame of the particle's azimuth, then rotate
         * back to the meridian plane */
        double gn = sqrt(1.0 + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]) / (c * c));
        double vr = up[0] / gn, vp = up[1] / gn, vz = up[2] / gn;
        double rho = l[0] * node_zr[2 * n3[0] + 1] + l[1] * node_zr[2 * n3[1] + 1]
                   + l[2] * node_zr[2 * n3[2] + 1];
        double x = rho + vr * dt, y = vp * dt;
        double rn = sqrt(x * x + y * y);
        if (rn > 0.0) {
            double cs = x / rn, sn = y / rn;
            double ur = cs * up[0] + sn * up[1];
            double uphi = -sn * up[0] + cs * up[1];
            up[0] = ur;
            up[1] = uphi;
        }
        u[3 * p] = up[0];
        u[3 * p + 1] = up[1];
        u[3 * p + 2] = up[2];
        double d[2] = {vz * dt, rn - rho};

        /* walk the straight meridian segment, splitting it at edge crossings */
        int entered = -1, alive = 1;
        for (int ncross = 0;; ncross++) {
            const double *g = grad + 6 * t;
            double dl[3], le[3];
            for (int k = 0; k < 3; k++) {
                dl[k] = g[2 * k] * d[0] + g[2 * k + 1] * d[1];
                le[k] = l[k] + dl[k];
            }
            int kx = -1;
            double sx = 2.0;
            for (int k = 0; k < 3; k++) {
                if (k == entered || !(le[k] < 0.0)) continue;
                double s = l[k] / (l[k] - le[k]);
                if (s < sx) { sx = s; kx = k; }
            }
            if (kx < 0) {
                /* endpoint inside t; a round-off negative on the entry edge is clamped */
                if (entered >= 0 && le[entered] < 0.0) {
                    le[entered] = 0.0;
                    int i = (entered + 1) % 3, j = (entered + 2) % 3;
                    double sum = le[i] + le[j];
                    le[i] /= sum;
                    le[j] /= sum;
                }
                deposit_segment(&m, t, l, le, wJ, J);
                for (int k = 0; k < 3; k++) l[k] = le[k];
                break;
            }
            /* crossing point on local edge kx */
            double lc[3];
            int i = (kx + 1) % 3, j = (kx + 2) % 3;
            lc[kx] = 0.0;
            lc[i] = l[i] + sx * dl[i];
            lc[j] = l[j] + sx * dl[j];
            double sum = lc[i] + lc[j];
            lc[i] /= sum;
            lc[j] /= sum;
            deposit_segment(&m, t, l, lc, wJ, J);
            ORACLE_ATOMIC counters[2]++;
            int nb = tri_nbr[3 * t + kx];
            int tag = tri_btag[3 * t + kx];
            if (nb < 0 && tag == TAG_AXIS) {
                /* the meridian segment stays at rho >= 0; stop on the axis */
                for (int k = 0; k < 3; k++) l[k] = lc[k];
                break;
            }
            if (nb < 0 || ncross + 1 >= max_cross) {
                /* absorbed at the wall (or walk cap reached): its charge leaves */
                const int32_t *nn = tri_nodes + 3 * t;
                for (int k = 0; k < 3; k++) ORACLE_ATOMIC Qabs[nn[k]] += q_src * lc[k];
                if (nb >= 0) ORACLE_ATOMIC counters[1]++;
                ORACLE_ATOMIC counters[0]++;
                alive = 0;
                break;
            }
            /* enter the neighbour: shared nodes keep their lambda, the third is 0 */
            const int32_t *nn = tri_nodes + 3 * nb;
            int gi = tri_nodes[3 * t + i], gj = tri_nodes[3 * t + j];
            double ln[3];
            int third = -1;
            for (int k = 0; k < 3; k++) {
                if (nn[k] == gi) ln[k] = lc[i];
                else if (nn[k] == gj) ln[k] = lc[j];
                else { ln[k] = 0.0; third = k; }
            }
            for (int k = 0; k < 3; k++) l[k] = ln[k];
            entered = third;
            d[0] *= (1.0 - sx);
            d[1] *= (1.0 - sx);
            t = nb;
        }
        if (alive) {
            const int32_t *nn = tri_nodes + 3 * t;
            for (int k = 0; k < 3; k++) ORACLE_ATOMIC Q[nn[k]] += q_src * l[k];
            tri[p] = t;
            lam[3 * p] = l[0];
            lam[3 * p + 1] = l[1];
            lam[3 * p + 2] = l[2];
        } else {
            tri[p] = -1;
        }
    }
    return 0;
}

/* Host threads the particle loop runs on (1 in the plain build). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. charge: Q_k += q_src * lambda_k for every live particle. */
int oracle_deposit_charge(const int32_t *tri_nodes, int64_t np, const int32_t *tri,
                          const double *lam, double q_src, double *Q)
{
    for (int64_t p = 0; p < np; p++) {
        int t = tri[p];
        if (t < 0) continue;
        for (int k = 0; k < 3; k++) Q[tri_nodes[3 * t + k]] += q_src * lam[3 * p + k];
    }
    return 0;
}
