/*
 * oracle.c -- plain, slow, FP64 CPU restatement of the explicit Eulerian
 * finite-volume update of Wallis, Barton & Nikiforakis, "A unified diffuse
 * interface method for the interaction of rigid bodies with elastoplastic
 * solids and multi-phase mixtures" (arXiv:2111.11806).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header
 * or table with the CUDA path; the product never calls it.
 *
 * Everything is written as plain loops over cells, pencils and faces in the
 * order the paper states the method, with no blocking or fusion:
 *   - conserved variables and non-conservative form ......... Sec. 2.1.1, Sec. 3 (eq:sys_vec_form)
 *   - Mie-Grueneisen closure, sound speed ..................... Sec. 2.1.2 (eq:MieGruneisenEOS)
 *   - ideal gas, Romenskii solid .............................. Sec. 2.1.3 (eq:Romenskii)
 *   - stiffened gas (water): the Mie-Grueneisen form with
 *     Gamma = gamma-1, e_ref = 0, p_ref = -gamma p_inf
 *   - mixture rules and mixture pressure ...................... Sec. 2.2
 *   - rigid field r and its evolution ......................... Sec. 2.3 (eq:revo)
 *   - spatial operator D(U), MUSCL-BVD-THINC, HLLC, upwind r
 *     flux, non-conservative terms, rigid-cell skip ........... Sec. 3.1 (eq:spat_op)
 *   - SSP-RK3 in the four-temporary form ...................... Sec. 3.1
 *   - rigid interface seeding (original variant) .............. Sec. 3.2 (boxed routine)
 *   - Youngs normal ........................................... Sec. 3.3
 * The readings taken where the paper is silent (limiter, THINC constants,
 * Riemann wave speeds, the solid Riemann solver, plastic relaxation, the
 * pressure-force sum and body motion, CFL formula) are listed with each
 * function below.
 *
 * Parity status of each part: pinned by the tests under tests/ that run
 * without a GPU (closed forms, invariants, exact Riemann solutions).
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OMAXV 24
#define OMAXM 3      /* materials per grid */

enum { MAT_IDEAL = 0, MAT_STIFFENED = 1, MAT_ROMENSKII = 2 };

typedef struct {
    int kind;
    double gamma, pinf;                         /* ideal / stiffened gas */
    double rho0, K0, G0, alpha, beta, Gamma0;   /* Romenskii solid */
    double sigY;                                /* yield stress (0 for fluids) */
    int jc;                                     /* 1: Johnson-Cook flow stress instead of sigY */
    double jc_c1, jc_c2, jc_c3, jc_n, jc_m;     /* Table 2 constants */
    double jc_tmelt, jc_cv;                     /* melting temperature, specific heat */
} omat;

typedef struct {
    int dim;
    int n[3];
    double lo[3], dx[3];
    int periodic[3];
    int nmat, solid, nv, nvar;
    int hist;                                   /* 1: equivalent plastic strain of every material */
    int iphi, iar, imom, iE, iV, ir, ih;        /* plane offsets (ih: history planes after r) */
    int vmap[9][2];                             /* stored V components -> (a,b) */
    omat mat[OMAXM];
    long ncell;
    double *U, *Un, *U1, *U3, *D, *W, *tmp;
    unsigned char *mask;
    double vr[3], xb[3], mass, force[3];
    int dynamic;
    double thinc_beta;
    int use_thinc;
    double phi_guard;
    int hllc_lm;        /* 1: low-Mach HLLC-LM dissipation in the star region */
    int seed_variant;   /* 0: original seeding, 1: Riemann-problem based (Sec. 3.2) */
    int normal_method;  /* 0: Youngs, 1: ELVIRA (2-D) (Sec. 3.3) */
    int probe_mode;     /* 0: stepped probe 1.0..4.0 dx, 1: fixed 1.5 dx (Sec. 3.2) */
    int seed_stages;    /* 1: the stage inputs U1, U3 are seeded too, before stages 2 and 3
                           [reading: Sec. 3.2 seeds the ghost region once per step, before
                           stage 1; seeding every stage input is the option] */
    int reflect[3][2];  /* reflective wall on the low / high side of direction d */
    double *seed_n;     /* normal used by the last seeding per cell (3 planes) */
} ostate;

/* ---------------------------------------------------------------- helpers */

static long cell_index(const ostate *s, int i, int j, int k)
{
    return (long)i + (long)s->n[0] * ((long)j + (long)s->n[1] * (long)k);
}

/* Halo mapping: transmissive boundaries copy the nearest interior cell (zero
 * gradient); periodic boundaries wrap. */
static int map_index(const ostate *s, int d, int i)
{
    int n = s->n[d];
    if (s->periodic[d]) {
        int m = i % n;
        return m < 0 ? m + n : m;
    }
    if (i < 0) return 0;
    if (i > n - 1) return n - 1;
    return i;
}

static double phi_clip(double f);

/* Reflective wall: the halo cell i < 0 mirrors cell -1-i, the halo cell
 * i > n-1 mirrors cell 2n-1-i (clamped to the grid when n < 3). */
static int mirror_index(int n, int i)
{
    int m = i < 0 ? -1 - i : 2 * n - 1 - i;
    if (m < 0) m = 0;
    if (m > n - 1) m = n - 1;
    return m;
}

static void mat_zero(double M[3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) M[a][b] = 0.0;
}

/* Stored V components of one cell -> full 3x3 tensor (absent components 0). */
static void vbar_unpack(const ostate *s, const double *q, double A[3][3])
{
    mat_zero(A);
    for (int c = 0; c < s->nv; c++) A[s->vmap[c][0]][s->vmap[c][1]] = q[s->iV + c];
}

static void vbar_pack(const ostate *s, double A[3][3], double *q)
{
    for (int c = 0; c < s->nv; c++) q[s->iV + c] = A[s->vmap[c][0]][s->vmap[c][1]];
}

/* ------------------------------------------- symmetric 3x3 eigen (Jacobi) */

/* Cyclic Jacobi rotations on a symmetric 3x3 matrix: B = Q diag(lam) Q^T
 * (columns of Q are eigenvectors).  Textbook algorithm; iterates until the
 * off-diagonal part is below 1e-15 of the Frobenius norm. */
void o_sym_eig3(const double Bin[9], double lam[3], double Qout[9])
{
    double a[3][3], q[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            a[i][j] = 0.5 * (Bin[3 * i + j] + Bin[3 * j + i]);
            q[i][j] = (i == j) ? 1.0 : 0.0;
        }
    double nrm = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) nrm += a[i][j] * a[i][j];
    nrm = sqrt(nrm);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (sqrt(off) <= 1e-15 * nrm || off == 0.0) break;
        for (int p = 0; p < 2; p++)
            for (int r = p + 1; r < 3; r++) {
                if (a[p][r] == 0.0) continue;
                double theta = (a[r][r] - a[p][p]) / (2.0 * a[p][r]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double sn = t * c;
                /* a <- J^T a J with J the rotation in the (p,r) plane */
                for (int k = 0; k < 3; k++) {
                    double akp = a[k][p], akr = a[k][r];
                    a[k][p] = c * akp - sn * akr;
                    a[k][r] = sn * akp + c * akr;
                }
                for (int k = 0; k < 3; k++) {
                    double apk = a[p][k], ark = a[r][k];
                    a[p][k] = c * apk - sn * ark;
                    a[r][k] = sn * apk + c * ark;
                }
                for (int k = 0; k < 3; k++) {
                    double qkp = q[k][p], qkr = q[k][r];
                    q[k][p] = c * qkp - sn * qkr;
                    q[k][r] = sn * qkp + c * qkr;
                }
            }
    }
    for (int i = 0; i < 3; i++) {
        lam[i] = a[i][i];
        for (int j = 0; j < 3; j++) Qout[3 * i + j] = q[i][j];
    }
}

/* Deviatoric Hencky strain dev(H) = ln V, with V the stretch of A (V^2 =
 * A A^T), Sec. 2.1.2.  Returns dev(H) and J^2 = tr(dev(H) dev(H)^T).  The mean
 * of the log-stretches is removed so that dev(H) is traceless even when
 * det(A) has drifted from 1 numerically. */
void o_vbar_log(const double A[9], double devH[9], double *J2, double lam_out[3], double Q_out[9])
{
    double B[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double sum = 0.0;
            for (int k = 0; k < 3; k++) sum += A[3 * i + k] * A[3 * j + k];
            B[3 * i + j] = sum;
        }
    double lam[3], Q[9];
    o_sym_eig3(B, lam, Q);
    double h[3], hm = 0.0;
    for (int k = 0; k < 3; k++) {
        h[k] = 0.5 * log(lam[k]);
        hm += h[k];
    }
    hm /= 3.0;
    double j2 = 0.0;
    for (int k = 0; k < 3; k++) {
        h[k] -= hm;
        j2 += h[k] * h[k];
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double sum = 0.0;
            for (int k = 0; k < 3; k++) sum += Q[3 * i + k] * h[k] * Q[3 * j + k];
            devH[3 * i + j] = sum;
        }
    *J2 = j2;
    if (lam_out)
        for (int k = 0; k < 3; k++) lam_out[k] = lam[k];
    if (Q_out)
        for (int k = 0; k < 9; k++) Q_out[k] = Q[k];
}

/* Left polar decomposition A = V R with V = sqrt(A A^T) symmetric positive
 * definite and R orthogonal. */
void o_polar(const double A[9], double V[9], double R[9])
{
    double B[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double sum = 0.0;
            for (int k = 0; k < 3; k++) sum += A[3 * i + k] * A[3 * j + k];
            B[3 * i + j] = sum;
        }
    double lam[3], Q[9];
    o_sym_eig3(B, lam, Q);
    double sq[3], isq[3];
    for (int k = 0; k < 3; k++) {
        sq[k] = sqrt(lam[k]);
        isq[k] = 1.0 / sq[k];
    }
    double Vinv[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s1 = 0.0, s2 = 0.0;
            for (int k = 0; k < 3; k++) {
                s1 += Q[3 * i + k] * sq[k] * Q[3 * j + k];
                s2 += Q[3 * i + k] * isq[k] * Q[3 * j + k];
            }
            V[3 * i + j] = s1;
            Vinv[3 * i + j] = s2;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double sum = 0.0;
            for (int k = 0; k < 3; k++) sum += Vinv[3 * i + k] * A[3 * k + j];
            R[3 * i + j] = sum;
        }
}

/* ---------------------------------------------------------- thermodynamics */

/* Reference curves of one material in the Mie-Grueneisen form
 * p = p_ref + rho Gamma (e - e_ref)  (Sec. 2.1.2, eq:MieGruneisenEOS).
 * out = {Gamma, e_ref, p_ref, de_ref/drho, dp_ref/drho, G}.
 *  ideal gas (Sec. 2.1.3): p_ref = e_ref = 0, Gamma = gamma - 1.
 *  stiffened gas: Gamma = gamma - 1, e_ref = 0, p_ref = -gamma p_inf.
 *  Romenskii (Sec. 2.1.3, eq:Romenskii, as printed with 1/rho in the cold
 *  term): e_ref = K0/(2 rho alpha^2) (x^alpha - 1)^2 + G J^2 / rho,
 *  G = G0 x^(beta+1), x = rho/rho0, p_ref = rho^2 de_ref/drho. */
void o_mat_ref(const omat *m, double rho, double J2, double out[6])
{
    if (m->kind == MAT_IDEAL) {
        out[0] = m->gamma - 1.0;
        out[1] = 0.0; out[2] = 0.0; out[3] = 0.0; out[4] = 0.0; out[5] = 0.0;
        return;
    }
    if (m->kind == MAT_STIFFENED) {
        out[0] = m->gamma - 1.0;
        out[1] = 0.0;
        out[2] = -m->gamma * m->pinf;
        out[3] = 0.0; out[4] = 0.0; out[5] = 0.0;
        return;
    }
    /* Romenskii */
    double al = m->alpha, be = m->beta, K0 = m->K0, rho0 = m->rho0;
    double x = rho / rho0;
    double xa = pow(x, al);
    double ec = K0 / (2.0 * rho * al * al) * (xa - 1.0) * (xa - 1.0);
    double pc = -K0 / (2.0 * al * al) * (xa - 1.0) * (xa - 1.0) + (K0 / al) * (xa - 1.0) * xa;
    double dpc = (K0 / rho0) * pow(x, al - 1.0) * (2.0 * xa - 1.0 - (xa - 1.0) / al);
    double G = m->G0 * pow(x, be + 1.0);
    double es = G * J2 / rho;
    double ps = be * G * J2;
    double dps = be * (be + 1.0) * G * J2 / rho;
    out[0] = m->Gamma0;
    out[1] = ec + es;
    out[2] = pc + ps;
    out[3] = (pc + ps) / (rho * rho);
    out[4] = dpc + dps;
    out[5] = G;
}

/* Full thermodynamic state of one cell or face, derived from primitives. */
typedef struct {
    double phi[OMAXM], rhol[OMAXM], ar[OMAXM];
    double rho, u[3], p, rhoE, c2, G, sigY;
    double devH[3][3], A[3][3], J2;
    double eps[OMAXM];  /* equivalent plastic strain of each material (history planes) */
} othermo;

/* Mixture closure from primitives (Sec. 2.2): rho = sum phi_l rho_l,
 * rho e = sum [phi_l rho_l e_ref,l + phi_l (p - p_ref,l)/Gamma_l],
 * G = sum(phi_l G_l/Gamma_l) / sum(phi_l/Gamma_l),
 * c^2 = sum(Y_l c_l^2/Gamma_l) / sum(phi_l/Gamma_l)  [reading of the printed
 * rule: Y_l carries the phi_l weight once, so the rule reduces to c_l for a
 * single material and for identical materials], c_l^2 = a_l^2 + 4/3 G_l/rho_l
 * (Sec. 2.1.2). */
static void thermo_from_prim(const ostate *s, const double *w, othermo *t)
{
    int N = s->nmat;
    double fsum = 0.0;
    for (int l = 0; l < N - 1; l++) {
        t->phi[l] = w[s->iphi + l];
        fsum += t->phi[l];
    }
    t->phi[N - 1] = 1.0 - fsum;
    t->rho = 0.0;
    for (int l = 0; l < N; l++) {
        t->phi[l] = phi_clip(t->phi[l]);
        t->rhol[l] = w[s->iar + l];
        t->ar[l] = t->phi[l] * t->rhol[l];
        t->rho += t->ar[l];
    }
    for (int a = 0; a < 3; a++) t->u[a] = (a < s->dim) ? w[s->imom + a] : 0.0;
    t->p = w[s->iE];
    for (int l = 0; l < N; l++) t->eps[l] = s->hist ? w[s->ih + l] : 0.0;
    mat_zero(t->devH);
    mat_zero(t->A);
    t->J2 = 0.0;
    if (s->solid) {
        double A9[9], dH[9];
        vbar_unpack(s, w, t->A);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) A9[3 * i + j] = t->A[i][j];
        o_vbar_log(A9, dH, &t->J2, NULL, NULL);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) t->devH[i][j] = dH[3 * i + j];
    }
    double rhoe = 0.0, den = 0.0, Gnum = 0.0, Ynum = 0.0, Snum = 0.0;
    for (int l = 0; l < N; l++) {
        double ref[6];
        o_mat_ref(&s->mat[l], t->rhol[l], t->J2, ref);
        double Gam = ref[0];
        /* a material with no mass carries no reference energy and no sound
         * speed weight (its phasic density may be 0 there) */
        if (t->ar[l] != 0.0) rhoe += t->ar[l] * ref[1];
        rhoe += t->phi[l] * (t->p - ref[2]) / Gam;
        den += t->phi[l] / Gam;
        Gnum += t->phi[l] * ref[5] / Gam;
        Snum += t->phi[l] * s->mat[l].sigY / Gam;
        double rl = t->rhol[l];
        double a2 = Gam * t->p / rl + (t->p - ref[2]) / rl + ref[4] - Gam * rl * ref[3];
        double c2l = a2 + 4.0 / 3.0 * ref[5] / rl;
        if (t->ar[l] != 0.0) Ynum += (t->ar[l] / t->rho) * c2l / Gam;
    }
    double ke = 0.0;
    for (int a = 0; a < 3; a++) ke += 0.5 * t->rho * t->u[a] * t->u[a];
    t->rhoE = rhoe + ke;
    t->G = Gnum / den;
    t->sigY = Snum / den;
    t->c2 = Ynum / den;
}

/* Volume fraction used as a closure weight: clipped to [0, 1] [reading; the
 * transported phi may leave the interval by round-off-sized amounts at
 * interfaces]. */
static double phi_clip(double f) { return f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f); }

/* Phasic density rho_l = (phi rho)_l / phi_l [Sec. 2.2].  Reading for a
 * material that is absent from the cell (clipped phi_l < 1e-6): its phasic
 * density is its reference density rho0 (when given), because the ratio of two
 * round-off-sized numbers carries no information and, through a stiff cold
 * curve, would set an arbitrary pressure. */
#define PHI_ABSENT 1e-6
static double phasic_density(const ostate *s, int l, double ar, double phc)
{
    if (phc < PHI_ABSENT && s->mat[l].rho0 > 0.0) return s->mat[l].rho0;
    return ar / (phc > s->phi_guard ? phc : s->phi_guard);
}

/* Conserved -> primitive (Sec. 2.2): phasic densities rho_l = (phi rho)_l /
 * phi_l (see phasic_density), velocity u = (rho u)/rho and
 * the mixture pressure
 * p = (rho e - sum_l [ (phi rho)_l e_ref,l - phi_l p_ref,l / Gamma_l ]) / sum_l phi_l/Gamma_l
 * with rho e = rho E - rho |u|^2 / 2. */
static void cons_to_prim(const ostate *s, const double *q, double *w)
{
    int N = s->nmat;
    double phi[OMAXM], ar[OMAXM], rho = 0.0, fsum = 0.0;
    for (int l = 0; l < N - 1; l++) {
        phi[l] = q[s->iphi + l];
        fsum += phi[l];
    }
    phi[N - 1] = 1.0 - fsum;
    for (int l = 0; l < N; l++) {
        ar[l] = q[s->iar + l];
        rho += ar[l];
    }
    double u[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < s->dim; a++) u[a] = q[s->imom + a] / rho;
    double J2 = 0.0;
    if (s->solid) {
        double A[3][3], A9[9], dH[9];
        vbar_unpack(s, q, A);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) A9[3 * i + j] = A[i][j];
        o_vbar_log(A9, dH, &J2, NULL, NULL);
    }
    double ke = 0.0;
    for (int a = 0; a < 3; a++) ke += 0.5 * rho * u[a] * u[a];
    double rhoe = q[s->iE] - ke;
    double num = rhoe, den = 0.0;
    double rhol[OMAXM];
    for (int l = 0; l < N; l++) {
        double phc = phi_clip(phi[l]);
        rhol[l] = (N == 1) ? rho : phasic_density(s, l, ar[l], phc);
        double ref[6];
        o_mat_ref(&s->mat[l], rhol[l], J2, ref);
        if (ar[l] != 0.0) num -= ar[l] * ref[1];
        num += phc * ref[2] / ref[0];
        den += phc / ref[0];
    }
    for (int l = 0; l < N - 1; l++) w[s->iphi + l] = phi[l];
    for (int l = 0; l < N; l++) w[s->iar + l] = rhol[l];
    for (int a = 0; a < s->dim; a++) w[s->imom + a] = u[a];
    w[s->iE] = num / den;
    for (int c = 0; c < s->nv; c++) w[s->iV + c] = q[s->iV + c];
    w[s->ir] = q[s->ir];
    /* history: the specific value eps_l = (phi rho eps)_l / (phi rho)_l, 0 where
     * the material has no mass */
    if (s->hist)
        for (int l = 0; l < N; l++) w[s->ih + l] = ar[l] != 0.0 ? q[s->ih + l] / ar[l] : 0.0;
}

static void prim_to_cons(const ostate *s, const double *w, double *q)
{
    othermo t;
    thermo_from_prim(s, w, &t);
    int N = s->nmat;
    for (int l = 0; l < N - 1; l++) q[s->iphi + l] = t.phi[l];
    for (int l = 0; l < N; l++) q[s->iar + l] = t.ar[l];
    for (int a = 0; a < s->dim; a++) q[s->imom + a] = t.rho * t.u[a];
    q[s->iE] = t.rhoE;
    for (int c = 0; c < s->nv; c++) q[s->iV + c] = w[s->iV + c];
    q[s->ir] = w[s->ir];
    if (s->hist)
        for (int l = 0; l < N; l++) q[s->ih + l] = t.ar[l] * t.eps[l];
}

/* ------------------------------------------------------ reconstruction */

/* van Leer (harmonic) limited slope [reading: the paper names MUSCL without
 * a limiter]: 2ab/(a+b) when a and b have the same sign, else 0. */
static double vanleer(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return 2.0 * a * b / (a + b);
}

/* THINC face values of cell i from (q_{i-1}, q_i, q_{i+1}) (Sec. 3.1, the
 * MUSCL-BVD-THINC scheme it cites).  The profile is
 *   q(x) = q_min + dq/2 (1 + theta tanh(beta (x - x_c))),  x in [0,1],
 * with x_c fixed by requiring the cell average of q(x) to equal q_i.  The
 * average of tanh over the cell is (1/beta) ln[cosh(beta(1-x_c))/cosh(beta x_c)],
 * so cosh(beta - y)/cosh(y) = exp(theta beta (2C - 1)) with y = beta x_c and
 * C = (q_i - q_min)/dq; expanding cosh(beta - y) gives
 *   tanh(y) = (cosh(beta) - exp(theta beta (2C-1))) / sinh(beta).
 * The face values are q(0) and q(1).  Applied only where the cell is
 * monotone, (q_{i+1}-q_i)(q_i-q_{i-1}) > 0, and 1e-8 < C < 1-1e-8 [reading];
 * otherwise returns 0 and the caller keeps the MUSCL values. */
int o_thinc(double qm, double q0, double qp, double beta, double *fm, double *fp)
{
    if ((qp - q0) * (q0 - qm) <= 0.0) return 0;
    double qmin = qm < qp ? qm : qp;
    double qmax = qm < qp ? qp : qm;
    double dq = qmax - qmin;
    double theta = (qp - qm) >= 0.0 ? 1.0 : -1.0;
    double C = (q0 - qmin) / dq;
    if (!(C > 1e-8 && C < 1.0 - 1e-8)) return 0;
    double B = exp(theta * beta * (2.0 * C - 1.0));
    double ty = (cosh(beta) - B) / sinh(beta);          /* tanh(beta x_c) */
    double tb = tanh(beta);
    /* q(0): tanh(-beta x_c) = -ty;  q(1): tanh(beta - beta x_c) by the
     * addition formula */
    double t0 = -ty;
    double t1 = (tb - ty) / (1.0 - tb * ty);
    *fm = qmin + 0.5 * dq * (1.0 + theta * t0);
    *fp = qmin + 0.5 * dq * (1.0 + theta * t1);
    return 1;
}

/* ----------------------------------------------------- Riemann solver */

/* Flux quantities of one face state in direction d. */
typedef struct {
    othermo t;
    double c, T;          /* sound speed, normal traction T = -sigma_dd */
    double U[OMAXV];      /* conserved state (thermodynamic part) */
    double F[OMAXV];      /* physical flux (thermodynamic part) */
} oface;

/* sigma = -p I + 2 G dev(H) (tension positive) [reading of Sec. 2.1.2 against
 * Sec. 2.4, which writes sigma_ij = -p delta_ij for the fluid].  Momentum flux
 * rho u_a u_d - sigma_ad, energy flux rho E u_d - u_a sigma_ad. */
static void face_state(const ostate *s, int d, const double *w, oface *f)
{
    thermo_from_prim(s, w, &f->t);
    othermo *t = &f->t;
    f->c = sqrt(t->c2);
    f->T = t->p - 2.0 * t->G * t->devH[d][d];
    int N = s->nmat;
    for (int l = 0; l < N; l++) {
        f->U[s->iar + l] = t->ar[l];
        f->F[s->iar + l] = t->ar[l] * t->u[d];
    }
    for (int a = 0; a < s->dim; a++) {
        double sig = -t->p * (a == d ? 1.0 : 0.0) + 2.0 * t->G * t->devH[a][d];
        f->U[s->imom + a] = t->rho * t->u[a];
        f->F[s->imom + a] = t->rho * t->u[a] * t->u[d] - sig;
    }
    double work = 0.0;
    for (int a = 0; a < 3; a++) {
        double sig = -t->p * (a == d ? 1.0 : 0.0) + 2.0 * t->G * t->devH[a][d];
        work += t->u[a] * sig;
    }
    f->U[s->iE] = t->rhoE;
    f->F[s->iE] = t->rhoE * t->u[d] - work;
    if (s->hist)
        for (int l = 0; l < N; l++) {
            f->U[s->ih + l] = t->ar[l] * t->eps[l];
            f->F[s->ih + l] = t->ar[l] * t->eps[l] * t->u[d];
        }
}

/* HLLC flux at a face in direction d (Sec. 3.1: Toro's HLLC for the
 * thermodynamic variables).  Readings: Davis wave-speed estimates
 * S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R); the
 * pressure of the fluid HLLC is replaced by the normal traction T = -sigma_dd
 * for solids (stands in for the HLLD of the full system); partial densities
 * scale like the mixture density in the star states.  Outputs:
 *   F[]     full flux vector (all nvar planes, r excluded -- set by caller),
 *   us[3]   face velocity u* of the state at x/t = 0 (normal: u_L, S* or u_R;
 *           tangential: upwind by S*, tie to the left),
 *   vrow[3] V*_{d b}, the row d of the upwind (by S*) face V. */
/* The value at x/t = 0 of a quantity carried by the contact: the left value
 * when S* > 0, the right one when S* < 0, and [reading] their mean when
 * S* = 0, so that the face of two mirror-image states (a wall) gets the
 * mirror-symmetric value. */
static double upwind(double Ss, double xl, double xr)
{
    return Ss > 0.0 ? xl : (Ss < 0.0 ? xr : 0.5 * (xl + xr));
}

void o_hllc(const ostate *s, int d, const double *wL, const double *wR, double *F, double us[3], double vrow[3])
{
    oface L, R;
    face_state(s, d, wL, &L);
    face_state(s, d, wR, &R);
    double uL = L.t.u[d], uR = R.t.u[d];
    double SL = fmin(uL - L.c, uR - R.c);
    double SR = fmax(uL + L.c, uR + R.c);
    double rL = L.t.rho, rR = R.t.rho;
    double Ss = (R.T - L.T + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    int N = s->nmat;
    /* thermodynamic variables */
    oface *K;
    double SK;
    int region; /* 0: F_L, 1: F*_L, 2: F*_R, 3: F_R */
    if (SL >= 0.0) region = 0;
    else if (Ss >= 0.0) region = 1;
    else if (SR > 0.0) region = 2;
    else region = 3;
    K = (region <= 1) ? &L : &R;
    SK = (region <= 1) ? SL : SR;
    /* the conserved planes the HLLC waves carry: partial densities, momenta,
     * energy, and the history planes */
    int adv[OMAXV], nadv = 0;
    for (int v = s->iar; v <= s->iE; v++) adv[nadv++] = v;
    if (s->hist)
        for (int l = 0; l < N; l++) adv[nadv++] = s->ih + l;
    /* tangential traction and velocity at the face: the linear shear-wave
     * Riemann problem, sigma -/+ Z u constant along the right/left shear
     * characteristics, Z = sqrt(rho G) [reading: the paper's HLLD resolves
     * shear waves; this keeps the traction continuous so that a gas (Z = 0)
     * transmits no shear].  Without shear stiffness on either side the
     * tangential velocity is taken upwind by S*. */
    double sig_t[3] = {0.0, 0.0, 0.0}, ut_star[3] = {0.0, 0.0, 0.0};
    double ZL = sqrt(L.t.rho * L.t.G), ZR = sqrt(R.t.rho * R.t.G);
    for (int a = 0; a < 3; a++) {
        if (a == d) continue;
        double sL = 2.0 * L.t.G * L.t.devH[a][d], sR = 2.0 * R.t.G * R.t.devH[a][d];
        if (ZL + ZR > 0.0) {
            sig_t[a] = (ZR * sL + ZL * sR + ZL * ZR * (R.t.u[a] - L.t.u[a])) / (ZL + ZR);
            ut_star[a] = (ZL * L.t.u[a] + ZR * R.t.u[a] + sR - sL) / (ZL + ZR);
        } else {
            sig_t[a] = 0.0;
            ut_star[a] = upwind(Ss, L.t.u[a], R.t.u[a]);
        }
    }
    if ((region == 1 || region == 2) && s->hllc_lm) {
        /* HLLC-LM [reading: the paper uses it for the cylinder test without
         * giving it; the published low-Mach form]: the centred HLLC flux
         *   F = (F_L + F_R)/2 + [phi S_L (U*_L - U_L) + |S*| (U*_L - U*_R) + phi S_R (U*_R - U_R)]/2
         * with phi = sin(min(1, Ma/0.1) pi/2), Ma = max(|u_L|/c_L, |u_R|/c_R) taken
         * with the velocity normal to the face;
         * phi = 1 is the HLLC flux.  Tangential tractions as below. */
        double Ma = fmax(fabs(uL) / L.c, fabs(uR) / R.c);
        double phi = sin(fmin(1.0, Ma / 0.1) * M_PI / 2.0);
        oface *side[2] = {&L, &R};
        double Sside[2] = {SL, SR};
        double Fa[2][OMAXV], Us[2][OMAXV];
        double work_ts = 0.0;
        for (int a = 0; a < 3; a++)
            if (a != d) work_ts += ut_star[a] * sig_t[a];
        for (int k = 0; k < 2; k++) {
            oface *Kk = side[k];
            double SKk = Sside[k], uKk = Kk->t.u[d];
            double chi = (SKk - uKk) / (SKk - Ss);
            for (int i = 0; i < nadv; i++) Fa[k][adv[i]] = Kk->F[adv[i]];
            double work_t = 0.0;
            for (int a = 0; a < 3; a++) {
                if (a == d) continue;
                double sK = 2.0 * Kk->t.G * Kk->t.devH[a][d];
                if (a < s->dim) Fa[k][s->imom + a] += sK;
                work_t += Kk->t.u[a] * sK;
            }
            Fa[k][s->iE] += work_t;
            for (int l = 0; l < N; l++) Us[k][s->iar + l] = Kk->t.ar[l] * chi;
            for (int a = 0; a < s->dim; a++) Us[k][s->imom + a] = Kk->t.rho * chi * (a == d ? Ss : Kk->t.u[a]);
            double EK = Kk->t.rhoE / Kk->t.rho;
            Us[k][s->iE] = Kk->t.rho * chi * (EK + (Ss - uKk) * (Ss + Kk->T / (Kk->t.rho * (SKk - uKk))));
            if (s->hist)
                for (int l = 0; l < N; l++) Us[k][s->ih + l] = Kk->t.ar[l] * Kk->t.eps[l] * chi;
        }
        for (int i = 0; i < nadv; i++) {
            const int v = adv[i];
            F[v] = 0.5 * (Fa[0][v] + Fa[1][v]) +
                   0.5 * (phi * SL * (Us[0][v] - L.U[v]) + fabs(Ss) * (Us[0][v] - Us[1][v]) +
                          phi * SR * (Us[1][v] - R.U[v]));
        }
        for (int a = 0; a < s->dim; a++)
            if (a != d) F[s->imom + a] -= sig_t[a];
        F[s->iE] -= work_ts;
    } else if (region == 0 || region == 3) {
        for (int i = 0; i < nadv; i++) F[adv[i]] = K->F[adv[i]];
    } else {
        /* HLLC on the advective part with the normal traction; the
         * tangential traction enters through its star value */
        double uK = K->t.u[d];
        double chi = (SK - uK) / (SK - Ss);
        double Us[OMAXV], Fa[OMAXV];
        for (int i = 0; i < nadv; i++) Fa[adv[i]] = K->F[adv[i]];
        double work_t = 0.0, work_ts = 0.0;
        for (int a = 0; a < 3; a++) {
            if (a == d) continue;
            double sK = 2.0 * K->t.G * K->t.devH[a][d];
            if (a < s->dim) Fa[s->imom + a] += sK;        /* remove -sigma_ad */
            work_t += K->t.u[a] * sK;
            work_ts += ut_star[a] * sig_t[a];
        }
        Fa[s->iE] += work_t;                              /* remove -u_t sigma_td */
        for (int l = 0; l < N; l++) Us[s->iar + l] = K->t.ar[l] * chi;
        for (int a = 0; a < s->dim; a++) Us[s->imom + a] = K->t.rho * chi * (a == d ? Ss : K->t.u[a]);
        double EK = K->t.rhoE / K->t.rho;
        Us[s->iE] = K->t.rho * chi * (EK + (Ss - uK) * (Ss + K->T / (K->t.rho * (SK - uK))));
        if (s->hist)
            for (int l = 0; l < N; l++) Us[s->ih + l] = K->t.ar[l] * K->t.eps[l] * chi;
        for (int i = 0; i < nadv; i++) F[adv[i]] = Fa[adv[i]] + SK * (Us[adv[i]] - K->U[adv[i]]);
        for (int a = 0; a < s->dim; a++)
            if (a != d) F[s->imom + a] -= sig_t[a];
        F[s->iE] -= work_ts;
    }
    /* interface state at x/t = 0 */
    for (int a = 0; a < 3; a++) us[a] = (region == 0 || region == 3) ? K->t.u[a] : ut_star[a];
    if (region == 0) us[d] = uL;
    else if (region == 3) us[d] = uR;
    else us[d] = Ss;
    /* volume fractions: phi* upwind by S*, conservative part phi* u*_d */
    for (int l = 0; l < N - 1; l++) F[s->iphi + l] = upwind(Ss, L.t.phi[l], R.t.phi[l]) * us[d];
    /* stretch tensor: F(V_ab) = V*_ab u*_d - V*_db u*_a */
    for (int b = 0; b < 3; b++) vrow[b] = upwind(Ss, L.t.A[d][b], R.t.A[d][b]);
    for (int c = 0; c < s->nv; c++) {
        int a = s->vmap[c][0], b = s->vmap[c][1];
        F[s->iV + c] = upwind(Ss, L.t.A[a][b], R.t.A[a][b]) * us[d] - vrow[b] * us[a];
    }
}

/* ------------------------------------------------------ spatial operator */

/* The mirror image of a primitive state in a wall normal to direction d:
 * velocity and stretch tensor transformed by the reflection P = I - 2 e_d e_d^T
 * (u_d changes sign; V_ab changes sign when exactly one of a, b is d); the
 * scalars are even. */
static void reflect_prim(const ostate *s, int d, double *w)
{
    w[s->imom + d] = -w[s->imom + d];
    for (int c = 0; c < s->nv; c++) {
        int a = s->vmap[c][0], b = s->vmap[c][1];
        if ((a == d) != (b == d)) w[s->iV + c] = -w[s->iV + c];
    }
}

/* D(U) of eq:spat_op (Sec. 3.1): for every direction d, the pencil of
 * primitives is reconstructed (MUSCL on all primitives; BVD-THINC on every
 * volume fraction and on r), the face fluxes are computed (HLLC; upwind r
 * flux with the body velocity), and
 *   D_i += (F_{i+1/2} - F_{i-1/2}) / dx_d - s_nc,i
 * with the non-conservative terms
 *   phi_l:  phi_l,i (u*_{d,R} - u*_{d,L}) / dx_d
 *   V_ab:   [2/3 V_ab,i (u*_{d,R} - u*_{d,L}) - u_a,i (V*_{db,R} - V*_{db,L})] / dx_d
 *   r:      r_i ((v_r)_{d,R} - (v_r)_{d,L}) / dx_d   (zero for a rigid translation)
 * where R is the face i+1/2 and L the face i-1/2. */
static void compute_D(ostate *s, const double *U, double *D)
{
    int nv = s->nvar;
    long nc = s->ncell;
    memset(D, 0, sizeof(double) * nv * nc);
    /* primitives of all cells */
    for (long c = 0; c < nc; c++) {
        double q[OMAXV] = {0.0}, w[OMAXV];
        for (int v = 0; v < nv; v++) q[v] = U[v * nc + c];
        cons_to_prim(s, q, w);
        for (int v = 0; v < nv; v++) s->W[v * nc + c] = w[v];
    }
    for (int d = 0; d < s->dim; d++) {
        int n = s->n[d];
        int e1 = (d == 0) ? 1 : 0;            /* the two other directions */
        int e2 = (d == 2) ? 1 : 2;
        int m1 = s->n[e1], m2 = s->n[e2];
        double *P = (double *)malloc(sizeof(double) * (n + 6) * nv);          /* cells -3..n+2 */
        double *Qm = (double *)malloc(sizeof(double) * (n + 6) * nv);         /* chosen face values */
        double *Qp = (double *)malloc(sizeof(double) * (n + 6) * nv);
        double *Mm = (double *)malloc(sizeof(double) * (n + 6) * nv);         /* MUSCL face values */
        double *Mp = (double *)malloc(sizeof(double) * (n + 6) * nv);
        double *Tm = (double *)malloc(sizeof(double) * (n + 6) * nv);         /* THINC face values */
        double *Tp = (double *)malloc(sizeof(double) * (n + 6) * nv);
        double *Ff = (double *)malloc(sizeof(double) * (n + 1) * nv);         /* face fluxes */
        double *Us = (double *)malloc(sizeof(double) * (n + 1) * 3);
        double *Vr = (double *)malloc(sizeof(double) * (n + 1) * 3);
        for (int j2 = 0; j2 < m2; j2++)
            for (int j1 = 0; j1 < m1; j1++) {
                /* gather the pencil with its halo of 3 */
                for (int i = -3; i < n + 3; i++) {
                    int idx[3];
                    int wall = (i < 0 && s->reflect[d][0]) || (i > n - 1 && s->reflect[d][1]);
                    idx[d] = wall ? mirror_index(n, i) : map_index(s, d, i);
                    idx[e1] = j1;
                    idx[e2] = j2;
                    long c = cell_index(s, idx[0], idx[1], idx[2]);
                    for (int v = 0; v < nv; v++) P[(i + 3) * nv + v] = s->W[v * nc + c];
                    if (wall) reflect_prim(s, d, &P[(i + 3) * nv]);
                }
                /* MUSCL and THINC face values of cells -2..n+1 */
                for (int i = -2; i < n + 2; i++) {
                    const double *qm = &P[(i + 2) * nv], *q0 = &P[(i + 3) * nv], *qp = &P[(i + 4) * nv];
                    for (int v = 0; v < nv; v++) {
                        double sl = vanleer(q0[v] - qm[v], qp[v] - q0[v]);
                        Mm[(i + 3) * nv + v] = q0[v] - 0.5 * sl;
                        Mp[(i + 3) * nv + v] = q0[v] + 0.5 * sl;
                        Tm[(i + 3) * nv + v] = Mm[(i + 3) * nv + v];
                        Tp[(i + 3) * nv + v] = Mp[(i + 3) * nv + v];
                    }
                    if (s->use_thinc) {
                        for (int v = 0; v < nv; v++) {
                            int isfrac = (v >= s->iphi && v < s->iphi + s->nmat - 1) || v == s->ir;
                            if (!isfrac) continue;
                            double fm, fp;
                            if (o_thinc(qm[v], q0[v], qp[v], s->thinc_beta, &fm, &fp)) {
                                Tm[(i + 3) * nv + v] = fm;
                                Tp[(i + 3) * nv + v] = fp;
                            }
                        }
                    }
                }
                /* BVD: per cell -1..n, keep THINC only if its total boundary
                 * variation is strictly lower than MUSCL's */
                for (int i = -1; i < n + 1; i++) {
                    for (int v = 0; v < nv; v++) {
                        int a = (i + 3) * nv + v, am = (i + 2) * nv + v, ap = (i + 4) * nv + v;
                        double tbvM = fabs(Mp[am] - Mm[a]) + fabs(Mp[a] - Mm[ap]);
                        double tbvT = fabs(Tp[am] - Tm[a]) + fabs(Tp[a] - Tm[ap]);
                        if (tbvT < tbvM) {
                            Qm[a] = Tm[a];
                            Qp[a] = Tp[a];
                        } else {
                            Qm[a] = Mm[a];
                            Qp[a] = Mp[a];
                        }
                    }
                }
                /* face fluxes, face f between cells f-1 and f */
                for (int f = 0; f <= n; f++) {
                    const double *wL = &Qp[(f - 1 + 3) * nv];
                    const double *wR = &Qm[(f + 3) * nv];
                    o_hllc(s, d, wL, wR, &Ff[f * nv], &Us[f * 3], &Vr[f * 3]);
                    double vd = s->vr[d];
                    double rf = 0.0;
                    if (vd > 0.0) rf = wL[s->ir] * vd;
                    else if (vd < 0.0) rf = wR[s->ir] * vd;
                    Ff[f * nv + s->ir] = rf;
                }
                /* divergence and non-conservative terms of cells 0..n-1 */
                for (int i = 0; i < n; i++) {
                    int idx[3];
                    idx[d] = i;
                    idx[e1] = j1;
                    idx[e2] = j2;
                    long c = cell_index(s, idx[0], idx[1], idx[2]);
                    const double *w = &P[(i + 3) * nv];
                    double inv = 1.0 / s->dx[d];
                    double dus = Us[(i + 1) * 3 + d] - Us[i * 3 + d];
                    for (int v = 0; v < nv; v++) {
                        double div = (Ff[(i + 1) * nv + v] - Ff[i * nv + v]) * inv;
                        double snc = 0.0;
                        if (v >= s->iphi && v < s->iphi + s->nmat - 1) snc = w[v] * dus * inv;
                        if (v >= s->iV && v < s->iV + s->nv) {
                            int cc = v - s->iV;
                            int a = s->vmap[cc][0], b = s->vmap[cc][1];
                            double ua = (a < s->dim) ? w[s->imom + a] : 0.0;
                            snc = (2.0 / 3.0 * w[v] * dus - ua * (Vr[(i + 1) * 3 + b] - Vr[i * 3 + b])) * inv;
                        }
                        if (v == s->ir) snc = w[v] * (s->vr[d] - s->vr[d]) * inv;
                        D[v * nc + c] += div - snc;
                    }
                }
            }
        free(P); free(Qm); free(Qp); free(Mm); free(Mp); free(Tm); free(Tp);
        free(Ff); free(Us); free(Vr);
    }
}

/* -------------------------------------------------------- rigid seeding */

static double cell_centre(const ostate *s, int d, int i)
{
    return s->lo[d] + (i + 0.5) * s->dx[d];
}

/* Central-difference gradient of r at cell (i,j,k) (Youngs, Sec. 3.3). */
static void grad_r(const ostate *s, const double *U, const int ijk[3], double g[3])
{
    long nc = s->ncell;
    for (int d = 0; d < 3; d++) {
        g[d] = 0.0;
        if (d >= s->dim) continue;
        int lo[3] = {ijk[0], ijk[1], ijk[2]}, hi[3] = {ijk[0], ijk[1], ijk[2]};
        lo[d] = map_index(s, d, ijk[d] - 1);
        hi[d] = map_index(s, d, ijk[d] + 1);
        double rW = U[s->ir * nc + cell_index(s, lo[0], lo[1], lo[2])];
        double rE = U[s->ir * nc + cell_index(s, hi[0], hi[1], hi[2])];
        g[d] = (rE - rW) / (2.0 * s->dx[d]);
    }
}

/* Riemann-problem-based seeding (Sec. 3.2, step 5, second option): the cell
 * takes the right star state of the HLLC problem along the normal n between
 * the reflected state (left) and the interpolated state (right), here solved
 * frame-free: normal velocity u.n, tangential velocity u - (u.n) n, normal
 * traction T = p - 2G n.devH.n, Davis wave speeds and the contact speed S* as
 * in o_hllc; the star state keeps the right state's volume fractions, stretch
 * tensor and tangential velocity.  wnew: reflected primitives, wint:
 * interpolated primitives; q: conserved output. */
static void riemann_seed(const ostate *s, const double nrm[3], const double *wnew, const double *wint, double *q)
{
    othermo tl, tr;
    thermo_from_prim(s, wnew, &tl);
    thermo_from_prim(s, wint, &tr);
    double unL = 0.0, unR = 0.0, TnL = 0.0, TnR = 0.0;
    for (int a = 0; a < 3; a++) {
        unL += tl.u[a] * nrm[a];
        unR += tr.u[a] * nrm[a];
        for (int b = 0; b < 3; b++) {
            TnL += nrm[a] * tl.devH[a][b] * nrm[b];
            TnR += nrm[a] * tr.devH[a][b] * nrm[b];
        }
    }
    TnL = tl.p - 2.0 * tl.G * TnL;
    TnR = tr.p - 2.0 * tr.G * TnR;
    double cL = sqrt(tl.c2), cR = sqrt(tr.c2);
    double SL = fmin(unL - cL, unR - cR), SR = fmax(unL + cL, unR + cR);
    double Ss = (TnR - TnL + tl.rho * unL * (SL - unL) - tr.rho * unR * (SR - unR)) /
                (tl.rho * (SL - unL) - tr.rho * (SR - unR));
    double chi = (SR - unR) / (SR - Ss);
    int N = s->nmat;
    for (int l = 0; l < N - 1; l++) q[s->iphi + l] = tr.phi[l];
    for (int l = 0; l < N; l++) q[s->iar + l] = tr.ar[l] * chi;
    double rs = tr.rho * chi;
    for (int a = 0; a < s->dim; a++) q[s->imom + a] = rs * (Ss * nrm[a] + (tr.u[a] - unR * nrm[a]));
    double ER = tr.rhoE / tr.rho;
    q[s->iE] = rs * (ER + (Ss - unR) * (Ss + TnR / (tr.rho * (SR - unR))));
    for (int c = 0; c < s->nv; c++) q[s->iV + c] = wint[s->iV + c];
    q[s->ir] = wint[s->ir];
    if (s->hist)
        for (int l = 0; l < N; l++) q[s->ih + l] = tr.ar[l] * chi * tr.eps[l];
}

/* ------------------------------------------------ ELVIRA normal (2-D) */

/* Fraction of the rectangle [x0, x0+hx] x [y0, y0+hy] lying on the side
 * nx x + ny y <= alpha of a line: the rectangle's polygon clipped by the
 * half-plane (one Sutherland-Hodgman pass), its area by the shoelace formula,
 * divided by hx hy. */
double o_cut_fraction(double nx, double ny, double alpha, double x0, double y0, double hx, double hy)
{
    double px[4] = {x0, x0 + hx, x0 + hx, x0}, py[4] = {y0, y0, y0 + hy, y0 + hy};
    double qx[8], qy[8];
    int nq = 0;
    for (int k = 0; k < 4; k++) {
        int kn = (k + 1) % 4;
        double dk = nx * px[k] + ny * py[k] - alpha;
        double dn = nx * px[kn] + ny * py[kn] - alpha;
        if (dk <= 0.0) {
            qx[nq] = px[k];
            qy[nq] = py[k];
            nq++;
        }
        if ((dk < 0.0 && dn > 0.0) || (dk > 0.0 && dn < 0.0)) {
            double t = dk / (dk - dn);
            qx[nq] = px[k] + t * (px[kn] - px[k]);
            qy[nq] = py[k] + t * (py[kn] - py[k]);
            nq++;
        }
    }
    double a2 = 0.0;
    for (int k = 0; k < nq; k++) {
        int kn = (k + 1) % nq;
        a2 += qx[k] * qy[kn] - qx[kn] * qy[k];
    }
    return fabs(0.5 * a2) / (hx * hy);
}

/* The line position alpha at which the rectangle holds the fraction f on the
 * side n.x <= alpha: bisection between the least and the largest n.x over
 * its corners, between which the fraction rises monotonically from 0 to 1. */
double o_cut_alpha(double nx, double ny, double f, double x0, double y0, double hx, double hy)
{
    double cx[4] = {x0, x0 + hx, x0 + hx, x0}, cy[4] = {y0, y0, y0 + hy, y0 + hy};
    double lo = nx * cx[0] + ny * cy[0], hi = lo;
    for (int k = 1; k < 4; k++) {
        double a = nx * cx[k] + ny * cy[k];
        lo = fmin(lo, a);
        hi = fmax(hi, a);
    }
    if (f <= 0.0) return lo;
    if (f >= 1.0) return hi;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (o_cut_fraction(nx, ny, mid, x0, y0, hx, hy) < f) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ELVIRA normal (Sec. 3.3; Pilliod & Puckett's method) of a cell from the
 * 3x3 block b[3 (l+1) + (k+1)] = r of cell (i+k, j+l), cell sizes hx, hy.
 * Candidate lines come from the two height functions of the block: the column
 * sums of r (interface height y as a function of x) and the row sums (x as a
 * function of y), each differenced backward, centrally and forward.  A column
 * slope m gives the normal (-m, s_y), a row slope m the normal (s_x, -m), with
 * s_y = -1 when the top row holds more r than the bottom row (else +1), s_x
 * likewise from the right and left columns, so that every candidate points
 * away from r = 1.  Each candidate line is placed to hold the centre cell's r;
 * the candidate whose line reproduces the nine values of r best (least sum of
 * squared differences) is returned as an outward unit normal.  [reading] An
 * earlier candidate wins ties within 1e-12, in the order central column,
 * central row, backward column, forward column, backward row, forward row. */
void o_elvira(const double b[9], double hx, double hy, double nrm[2])
{
    double h[3], g[3];
    for (int k = 0; k < 3; k++) h[k] = (b[k] + b[3 + k] + b[6 + k]) * hy;
    for (int l = 0; l < 3; l++) g[l] = (b[3 * l] + b[3 * l + 1] + b[3 * l + 2]) * hx;
    double sy = (g[2] > g[0]) ? -1.0 : 1.0;
    double sx = (h[2] > h[0]) ? -1.0 : 1.0;
    double mcol[3] = {(h[2] - h[0]) / (2.0 * hx), (h[1] - h[0]) / hx, (h[2] - h[1]) / hx};
    double mrow[3] = {(g[2] - g[0]) / (2.0 * hy), (g[1] - g[0]) / hy, (g[2] - g[1]) / hy};
    double cand[6][2] = {{-mcol[0], sy}, {sx, -mrow[0]}, {-mcol[1], sy},
                         {-mcol[2], sy}, {sx, -mrow[1]}, {sx, -mrow[2]}};
    double best = 0.0;
    for (int c = 0; c < 6; c++) {
        double len = sqrt(cand[c][0] * cand[c][0] + cand[c][1] * cand[c][1]);
        double nx = cand[c][0] / len, ny = cand[c][1] / len;
        double alpha = o_cut_alpha(nx, ny, b[4], -0.5 * hx, -0.5 * hy, hx, hy);
        double err = 0.0;
        for (int l = 0; l < 3; l++)
            for (int k = 0; k < 3; k++) {
                double f = o_cut_fraction(nx, ny, alpha, (k - 1.5) * hx, (l - 1.5) * hy, hx, hy);
                err += (f - b[3 * l + k]) * (f - b[3 * l + k]);
            }
        if (c == 0 || err < best - 1e-12) {
            best = err;
            nrm[0] = nx;
            nrm[1] = ny;
        }
    }
}

/* The rigid seeding routine (Sec. 3.2, boxed routine), applied once at the
 * start of the step to the state U0 it starts from:
 *  1. in every cell with r > 0.5, the outward normal: Youngs, n = -grad r/|grad r|
 *     with central differences, or (2-D option) the ELVIRA normal of the 3x3
 *     block of r; cells with |grad r| dx_min <= 1e-10 are left alone [reading];
 *  2. the probe point, stepped or fixed:
 *     stepped: s = 1.0, 1.5, ..., 4.0 dx_min along n [reading: step dx/2]; the
 *     first point whose 2^dim enclosing cell centres all lie in the domain (or
 *     wrap, for periodic directions) and have r < 0.5 is taken, a point
 *     within PROBE_SNAP cells of a cell-centre line counting as on it (the
 *     corners beyond carry no weight); no valid point -> the cell is unchanged;
 *     fixed: s = 1.5 dx_min, enclosing cells clamped into the domain (wrapped
 *     if periodic), whatever their r [reading];
 *     the primitives of U0 are interpolated multilinearly at the point;
 *  3-5. reflection in the frame of n, written frame-free with the Householder
 *     matrix P = I - 2 n n^T (R P R^T = diag(-1,1,1) in the rotated frame):
 *     u_new = P u_int + 2 (v_r . n) n,  V_new = P V_int P; scalars are copied;
 *     the original variant puts the new state in the cell (r is kept), the
 *     Riemann-problem variant the right HLLC star state of (new, interpolated).
 * Every seeded state is computed from U0 alone [reading: all cells seeded at
 * once], so the result does not depend on the loop order. */
/* A probe point within PROBE_SNAP cell widths of a cell-centre line is
 * taken to lie on it: the corners beyond the line get weight 0 and are not
 * part of the stencil (neither tested nor read) [reading: the paper's stencil
 * is the set of cells the interpolated state is made of; on a symmetry axis
 * the normal is axis-aligned, the probe steps are whole and half cells, and
 * the probe point falls exactly on a cell-centre line, where a zero-weight
 * corner would otherwise decide the step by the sign of a rounding error]. */
#define PROBE_SNAP 1e-3

void o_seed(ostate *s)
{
    long nc = s->ncell;
    int nv = s->nvar;
    double dxmin = s->dx[0];
    for (int d = 1; d < s->dim; d++) dxmin = fmin(dxmin, s->dx[d]);
    double *U0 = (double *)malloc(sizeof(double) * nv * nc);
    memcpy(U0, s->U, sizeof(double) * nv * nc);
    memset(s->seed_n, 0, sizeof(double) * 3 * nc);
    for (int k = 0; k < s->n[2]; k++)
        for (int j = 0; j < s->n[1]; j++)
            for (int i = 0; i < s->n[0]; i++) {
                long c = cell_index(s, i, j, k);
                if (!(U0[s->ir * nc + c] > 0.5)) continue;
                int ijk[3] = {i, j, k};
                double g[3];
                grad_r(s, U0, ijk, g);
                double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                if (!(gn * dxmin > 1e-10)) continue;
                double nrm[3] = {-g[0] / gn, -g[1] / gn, -g[2] / gn};
                if (s->normal_method == 1 && s->dim == 2) {
                    double blk[9], n2[2];
                    for (int l = -1; l <= 1; l++)
                        for (int m = -1; m <= 1; m++)
                            blk[3 * (l + 1) + (m + 1)] =
                                U0[s->ir * nc + cell_index(s, map_index(s, 0, i + m), map_index(s, 1, j + l), 0)];
                    o_elvira(blk, s->dx[0], s->dx[1], n2);
                    nrm[0] = n2[0];
                    nrm[1] = n2[1];
                    nrm[2] = 0.0;
                }
                int found = 0;
                double wint[OMAXV];
                int nsteps = s->probe_mode == 1 ? 1 : 7;
                for (int step = 0; step < nsteps && !found; step++) {
                    double sdist = (s->probe_mode == 1 ? 1.5 : 1.0 + 0.5 * step) * dxmin;
                    int base[3];
                    double frac[3];
                    for (int d = 0; d < 3; d++) {
                        base[d] = 0;
                        frac[d] = 0.0;
                        if (d >= s->dim) continue;
                        double xp = cell_centre(s, d, ijk[d]) + sdist * nrm[d];
                        double fi = (xp - s->lo[d]) / s->dx[d] - 0.5;
                        double fl = floor(fi);
                        double fr = fi - fl;
                        /* within PROBE_SNAP cells of a cell-centre line: on it */
                        if (fr < PROBE_SNAP) {
                            fr = 0.0;
                        } else if (fr > 1.0 - PROBE_SNAP) {
                            fr = 0.0;
                            fl += 1.0;
                        }
                        base[d] = (int)fl;
                        frac[d] = fr;
                    }
                    int ncorner = 1 << s->dim;
                    int ok = 1;
                    long cidx[8];
                    double wts[8];
                    for (int m = 0; m < ncorner && ok; m++) {
                        int ci[3] = {0, 0, 0};
                        double wt = 1.0;
                        int inside = 1;
                        for (int d = 0; d < s->dim; d++) {
                            int bit = (m >> d) & 1;
                            int ii = base[d] + bit;
                            if (!s->periodic[d] && (ii < 0 || ii > s->n[d] - 1)) inside = 0;
                            ci[d] = map_index(s, d, ii);
                            wt *= bit ? frac[d] : (1.0 - frac[d]);
                        }
                        long cc = cell_index(s, ci[0], ci[1], ci[2]);
                        /* the stepped probe needs fluid cells inside the domain;
                         * a corner of weight 0 (a probe point on a cell-centre
                         * line) is not part of the stencil */
                        if (s->probe_mode == 0 && wt > 0.0 && (!inside || !(U0[s->ir * nc + cc] < 0.5))) ok = 0;
                        cidx[m] = cc;
                        wts[m] = wt;
                    }
                    if (!ok) continue;
                    for (int v = 0; v < nv; v++) wint[v] = 0.0;
                    for (int m = 0; m < ncorner; m++) {
                        double q[OMAXV], w[OMAXV];
                        if (wts[m] == 0.0) continue;
                        for (int v = 0; v < nv; v++) q[v] = U0[v * nc + cidx[m]];
                        cons_to_prim(s, q, w);
                        for (int v = 0; v < nv; v++) wint[v] += wts[m] * w[v];
                    }
                    found = 1;
                }
                if (!found) continue;
                for (int d = 0; d < 3; d++) s->seed_n[d * nc + c] = nrm[d];
                double wref[OMAXV];     /* the interpolated state, before reflection */
                for (int v = 0; v < nv; v++) wref[v] = wint[v];
                wref[s->ir] = U0[s->ir * nc + c];
                /* reflect */
                double P[3][3];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) P[a][b] = (a == b ? 1.0 : 0.0) - 2.0 * nrm[a] * nrm[b];
                double u[3] = {0.0, 0.0, 0.0}, un[3];
                for (int a = 0; a < s->dim; a++) u[a] = wint[s->imom + a];
                double vn = s->vr[0] * nrm[0] + s->vr[1] * nrm[1] + s->vr[2] * nrm[2];
                for (int a = 0; a < 3; a++) {
                    un[a] = 2.0 * vn * nrm[a];
                    for (int b = 0; b < 3; b++) un[a] += P[a][b] * u[b];
                }
                for (int a = 0; a < s->dim; a++) wint[s->imom + a] = un[a];
                if (s->solid) {
                    double A[3][3], B[3][3], C[3][3];
                    vbar_unpack(s, wint, A);
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) {
                            double sum = 0.0;
                            for (int m = 0; m < 3; m++) sum += P[a][m] * A[m][b];
                            B[a][b] = sum;
                        }
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) {
                            double sum = 0.0;
                            for (int m = 0; m < 3; m++) sum += B[a][m] * P[m][b];
                            C[a][b] = sum;
                        }
                    vbar_pack(s, C, wint);
                }
                wint[s->ir] = U0[s->ir * nc + c];
                double q[OMAXV];
                if (s->seed_variant == 1) riemann_seed(s, nrm, wint, wref, q);
                else prim_to_cons(s, wint, q);
                for (int v = 0; v < nv; v++) s->U[v * nc + c] = q[v];
            }
    free(U0);
}

/* Pressure force on the body [not in the paper, which imposes v_r (Sec. 2.3);
 * reading]: F = sum_i p_i (grad r)_i dV over all cells, with the Youngs
 * central differences; it is the discrete form of -(surface integral of
 * p n_out dA).  Evaluated on the state after seeding. */
void o_force(ostate *s, double F[3])
{
    long nc = s->ncell;
    double dV = 1.0;
    for (int d = 0; d < s->dim; d++) dV *= s->dx[d];
    F[0] = F[1] = F[2] = 0.0;
    for (int k = 0; k < s->n[2]; k++)
        for (int j = 0; j < s->n[1]; j++)
            for (int i = 0; i < s->n[0]; i++) {
                long c = cell_index(s, i, j, k);
                int ijk[3] = {i, j, k};
                double g[3], q[OMAXV], w[OMAXV];
                grad_r(s, s->U, ijk, g);
                for (int v = 0; v < s->nvar; v++) q[v] = s->U[v * nc + c];
                cons_to_prim(s, q, w);
                for (int d = 0; d < 3; d++) F[d] += w[s->iE] * g[d] * dV;
            }
}

/* ------------------------------------------------------ plastic update */

/* Johnson-Cook flow stress of one material [readings: Table 2 gives the
 * constants c1, c2, c3, n, m, T_melt and C_V of copper but not the law; the
 * usual Johnson-Cook form is taken with the reference temperature JC_T0 and
 * the reference plastic strain rate JC_RATE0]:
 *   sigma_Y = (c1 + c2 eps^n) (1 + c3 ln max(rate/JC_RATE0, 1)) (1 - T*^m),
 *   T* = (T - JC_T0)/(T_melt - JC_T0) clipped to [0, 1]. */
#define JC_T0 298.0
#define JC_RATE0 1.0

static double jc_yield(const omat *m, double eps, double rate, double T)
{
    double ts = (T - JC_T0) / (m->jc_tmelt - JC_T0);
    ts = ts < 0.0 ? 0.0 : (ts > 1.0 ? 1.0 : ts);
    double r = rate / JC_RATE0;
    double e = eps > 0.0 ? eps : 0.0;
    return (m->jc_c1 + m->jc_c2 * pow(e, m->jc_n)) * (1.0 + m->jc_c3 * log(r > 1.0 ? r : 1.0)) *
           (1.0 - pow(ts, m->jc_m));
}

/* Temperature of material l [reading: the thermal part of its
 * Mie-Grueneisen energy over the specific heat, T = JC_T0 + (e - e_ref)/C_V
 * with e - e_ref = (p - p_ref)/(rho_l Gamma_l) at the cell's pressure]. */
static double jc_temperature(const omat *m, double p, double rhol, const double ref[6])
{
    return JC_T0 + (p - ref[2]) / (rhol * ref[0] * m->jc_cv);
}

/* Mixture yield stress of a cell for the return (Sec. 2.2 weights phi_l/Gamma_l),
 * with Johnson-Cook materials at the cell's plastic-strain rate `rate`. */
static double yield_mixture(const ostate *s, const othermo *t, double rate)
{
    double num = 0.0, den = 0.0;
    for (int l = 0; l < s->nmat; l++) {
        double ref[6];
        o_mat_ref(&s->mat[l], t->rhol[l], t->J2, ref);
        double sy = s->mat[l].sigY;
        if (s->mat[l].jc) sy = jc_yield(&s->mat[l], t->eps[l], rate, jc_temperature(&s->mat[l], t->p, t->rhol[l], ref));
        num += t->phi[l] * sy / ref[0];
        den += t->phi[l] / ref[0];
    }
    return num / den;
}

/* Perfect plasticity by instantaneous radial return [reading; Sec. 2.1.1
 * defers the convex-potential closure to Barton 2019]: the stretch is
 * re-symmetrised by the left polar decomposition A = V R (A A^T = Q diag(lam) Q^T),
 * the deviatoric log-stretches d_k = ln sqrt(lam_k) - mean are scaled by
 * s = min(1, sigma_Y/sigma_vm), sigma_vm = sqrt(3/2) 2 G |d|, with the mixture
 * G and sigma_Y weighted like the shear-modulus rule (Sec. 2.2), and
 * V <- Q diag(exp(s d_k)) Q^T (unimodular).  rho E, phi and phi rho are kept,
 * so the released shear energy becomes heat.  With Johnson-Cook materials the
 * yield stress depends on the plastic strain, the temperature and the
 * plastic-strain rate [reading: one explicit predictor; the rate is the
 * equivalent plastic strain a return at the rate-free yield stress would
 * remove, over the step dt (0 when dt = 0)]. */
static void plastic_cell(const ostate *s, double *q, double dt)
{
    double w[OMAXV];
    cons_to_prim(s, q, w);
    othermo t;
    thermo_from_prim(s, w, &t);
    double A9[9], dH[9], lam[3], Q[9], J2;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) A9[3 * i + j] = t.A[i][j];
    o_vbar_log(A9, dH, &J2, lam, Q);
    double h[3], hm = 0.0;
    for (int k = 0; k < 3; k++) {
        h[k] = 0.5 * log(lam[k]);
        hm += h[k];
    }
    hm /= 3.0;
    double nd = 0.0;
    for (int k = 0; k < 3; k++) {
        h[k] -= hm;
        nd += h[k] * h[k];
    }
    nd = sqrt(nd);
    double svm = sqrt(1.5) * 2.0 * t.G * nd;
    double sigY = t.sigY;
    int any_jc = 0;
    for (int l = 0; l < s->nmat; l++) any_jc |= s->mat[l].jc;
    if (any_jc) {
        double sy0 = yield_mixture(s, &t, 0.0);
        double rate = (svm > sy0 && dt > 0.0) ? sqrt(2.0 / 3.0) * (1.0 - sy0 / svm) * nd / dt : 0.0;
        sigY = yield_mixture(s, &t, rate);
    }
    double sc = (svm > sigY) ? sigY / svm : 1.0;
    /* equivalent plastic strain [reading: Sec. 2.1.1 names the history
     * variable without its evolution law]: the deviatoric log-strain removed
     * by the return, (1 - s) |d|, as the von Mises equivalent
     * sqrt(2/3) (1 - s) |d|, added to every material with a yield stress */
    if (s->hist && sc < 1.0) {
        double deps = sqrt(2.0 / 3.0) * (1.0 - sc) * nd;
        for (int l = 0; l < s->nmat; l++)
            if (s->mat[l].sigY > 0.0 || s->mat[l].jc) q[s->ih + l] += q[s->iar + l] * deps;
    }
    double Vn[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double sum = 0.0;
            for (int k = 0; k < 3; k++) sum += Q[3 * i + k] * exp(sc * h[k]) * Q[3 * j + k];
            Vn[i][j] = sum;
        }
    vbar_pack(s, Vn, q);
}

void o_plastic(ostate *s, double dt)
{
    if (!s->solid) return;
    long nc = s->ncell;
    for (long c = 0; c < nc; c++) {
        if (s->mask && s->mask[c]) continue;
        double q[OMAXV];
        for (int v = 0; v < s->nvar; v++) q[v] = s->U[v * nc + c];
        plastic_cell(s, q, dt);
        for (int v = 0; v < s->nvar; v++) s->U[v * nc + c] = q[v];
    }
}

/* ----------------------------------------------------- time step, RK */

/* dt = CFL / max_i sum_d (|u_d| + c)/dx_d over all cells, also covering the
 * body speed sum_d |v_r,d|/dx_d [reading: the paper takes a fraction of the
 * global maximum stable step without a formula]. */
double o_compute_dt(ostate *s, double cfl)
{
    long nc = s->ncell;
    double smax = 0.0;
    int bad = 0;
    for (long c = 0; c < nc; c++) {
        double q[OMAXV], w[OMAXV];
        othermo t;
        for (int v = 0; v < s->nvar; v++) q[v] = s->U[v * nc + c];
        cons_to_prim(s, q, w);
        thermo_from_prim(s, w, &t);
        double cs = sqrt(t.c2);
        double sum = 0.0;
        for (int d = 0; d < s->dim; d++) sum += (fabs(t.u[d]) + cs) / s->dx[d];
        if (sum != sum) bad = 1;
        else if (sum > smax) smax = sum;
    }
    if (bad) return NAN;
    double sb = 0.0;
    for (int d = 0; d < s->dim; d++) sb += fabs(s->vr[d]) / s->dx[d];
    if (sb > smax) smax = sb;
    return cfl / smax;
}

static int is_thermo(const ostate *s, int v) { return v != s->ir; }

/* One step: seeding (Sec. 3.2, once, before the hyperbolic update), the
 * pressure force on the seeded state, then the SSP-RK3 scheme of Sec. 3.1
 *   U1 = Un - dt D(Un);  U2 = U1 - dt D(U1);  U3 = 3/4 Un + 1/4 U2;
 *   U4 = U3 - dt D(U3);  U^{n+1} = 1/3 Un + 2/3 U4,
 * where the thermodynamic variables of cells with r^n > 0.5 are carried
 * unchanged (Sec. 3.1: rigid cells are not updated; they are re-seeded next
 * step) and r is updated everywhere.  Then plastic relaxation (solids) and
 * the body update v += dt F/m, x += dt v (dynamic body only). */
void o_step(ostate *s, double dt)
{
    long nc = s->ncell;
    int nv = s->nvar;
    o_seed(s);
    o_force(s, s->force);
    memcpy(s->Un, s->U, sizeof(double) * nv * nc);
    for (long c = 0; c < nc; c++) s->mask[c] = s->Un[s->ir * nc + c] > 0.5;
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    double *in[3] = {s->Un, s->U1, s->U3};
    double *out[3] = {s->U1, s->U3, s->U};
    for (int st = 0; st < 3; st++) {
        if (st > 0 && s->seed_stages) {
            /* the stage input's rigid band from its own fluid cells (the
             * mask and the force stay those of the step-start state) */
            double *keep = s->U;
            s->U = in[st];
            o_seed(s);
            s->U = keep;
        }
        compute_D(s, in[st], s->D);
        for (int v = 0; v < nv; v++)
            for (long c = 0; c < nc; c++) {
                long a = v * nc + c;
                if (s->mask[c] && is_thermo(s, v)) {
                    out[st][a] = s->Un[a];
                    continue;
                }
                double y = in[st][a] - dt * s->D[a];
                out[st][a] = (st == 0) ? y : ca[st] * s->Un[a] + cb[st] * y;
            }
    }
    o_plastic(s, dt);
    if (s->dynamic && s->mass > 0.0) {
        for (int d = 0; d < 3; d++) {
            s->vr[d] += dt * s->force[d] / s->mass;
            s->xb[d] += dt * s->vr[d];
        }
    }
}

/* ---------------------------------------------------------------- API */

/* solid: 0 fluids, 1 elastoplastic (stretch tensor planes), 2 elastoplastic
 * with one equivalent-plastic-strain plane (phi rho eps)_l per material after
 * r (Sec. 2.1.1 history variables). */
void *o_create(int dim, const int n[3], const double lo[3], const double hi[3], const int periodic[3], int nmat, int solid)
{
    if (nmat < 1 || nmat > OMAXM) return NULL;
    ostate *s = (ostate *)calloc(1, sizeof(ostate));
    s->dim = dim;
    s->ncell = 1;
    for (int d = 0; d < 3; d++) {
        s->n[d] = (d < dim) ? n[d] : 1;
        s->lo[d] = (d < dim) ? lo[d] : 0.0;
        s->dx[d] = (d < dim) ? (hi[d] - lo[d]) / n[d] : 1.0;
        s->periodic[d] = (d < dim) ? periodic[d] : 0;
        s->ncell *= s->n[d];
    }
    s->nmat = nmat;
    s->solid = solid != 0;
    s->hist = solid == 2;
    s->nv = solid ? (dim == 1 ? 3 : dim == 2 ? 5 : 9) : 0;
    s->iphi = 0;
    s->iar = nmat - 1;
    s->imom = 2 * nmat - 1;
    s->iE = s->imom + dim;
    s->iV = s->iE + 1;
    s->ir = s->iV + s->nv;
    s->ih = s->ir + 1;
    s->nvar = s->ih + (s->hist ? nmat : 0);
    if (dim == 1) {
        int m[3][2] = {{0, 0}, {1, 1}, {2, 2}};
        memcpy(s->vmap, m, sizeof(m));
    } else if (dim == 2) {
        int m[5][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}, {2, 2}};
        memcpy(s->vmap, m, sizeof(m));
    } else {
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                s->vmap[3 * a + b][0] = a;
                s->vmap[3 * a + b][1] = b;
            }
    }
    size_t sz = sizeof(double) * s->nvar * s->ncell;
    s->U = (double *)calloc(1, sz);
    s->Un = (double *)calloc(1, sz);
    s->U1 = (double *)calloc(1, sz);
    s->U3 = (double *)calloc(1, sz);
    s->D = (double *)calloc(1, sz);
    s->seed_n = (double *)calloc(3 * (size_t)s->ncell, sizeof(double));
    s->W = (double *)calloc(1, sz);
    s->mask = (unsigned char *)calloc(s->ncell, 1);
    s->thinc_beta = 1.6;
    s->use_thinc = 1;
    s->phi_guard = 1e-14;
    return s;
}

void o_destroy(void *h)
{
    ostate *s = (ostate *)h;
    if (!s) return;
    free(s->U); free(s->Un); free(s->U1); free(s->U3); free(s->D); free(s->W); free(s->mask); free(s->seed_n);
    free(s);
}

int o_nvar(void *h) { return ((ostate *)h)->nvar; }

void o_set_material(void *h, int l, int kind, double gamma, double pinf, double rho0, double K0, double G0,
                    double alpha, double beta, double Gamma0, double sigY)
{
    ostate *s = (ostate *)h;
    omat *m = &s->mat[l];
    m->kind = kind; m->gamma = gamma; m->pinf = pinf; m->rho0 = rho0; m->K0 = K0; m->G0 = G0;
    m->alpha = alpha; m->beta = beta; m->Gamma0 = Gamma0; m->sigY = sigY;
}

void o_set_options(void *h, int use_thinc, double thinc_beta)
{
    ostate *s = (ostate *)h;
    s->use_thinc = use_thinc;
    s->thinc_beta = thinc_beta;
}

void o_set_variants(void *h, int hllc_lm, int seed_variant, int normal_method, int probe_mode)
{
    ostate *s = (ostate *)h;
    s->hllc_lm = hllc_lm;
    s->seed_variant = seed_variant;
    s->normal_method = normal_method;
    s->probe_mode = probe_mode;
}

/* Seeding of every stage input (1) or of the step-start state only (0). */
void o_set_seed_stages(void *h, int on) { ((ostate *)h)->seed_stages = on != 0; }

/* The conserved planes of a stage input of the last step: k = 1 the input of
 * stage 2 (U1), k = 2 that of stage 3 (U3), as the stage read them (seeded
 * when the option is on). */
void o_get_stage_input(void *h, int k, double *out)
{
    ostate *s = (ostate *)h;
    memcpy(out, k == 1 ? s->U1 : s->U3, sizeof(double) * s->nvar * s->ncell);
}

/* Reflective walls: refl[2 d] / refl[2 d + 1] for the low / high side of a
 * non-periodic direction d. */
void o_set_walls(void *h, const int refl[6])
{
    ostate *s = (ostate *)h;
    for (int d = 0; d < 3; d++)
        for (int e = 0; e < 2; e++) s->reflect[d][e] = (d < s->dim && !s->periodic[d]) ? (refl[2 * d + e] != 0) : 0;
}

/* The normal each cell used in the last seeding (3 planes; 0 where the cell
 * was not seeded). */
void o_seed_normals(void *h, double *out)
{
    ostate *s = (ostate *)h;
    memcpy(out, s->seed_n, sizeof(double) * 3 * (size_t)s->ncell);
}

void o_set_prim(void *h, const double *prim)
{
    ostate *s = (ostate *)h;
    long nc = s->ncell;
    for (long c = 0; c < nc; c++) {
        double w[OMAXV], q[OMAXV];
        for (int v = 0; v < s->nvar; v++) w[v] = prim[v * nc + c];
        prim_to_cons(s, w, q);
        for (int v = 0; v < s->nvar; v++) s->U[v * nc + c] = q[v];
    }
}

void o_get_prim(void *h, double *prim)
{
    ostate *s = (ostate *)h;
    long nc = s->ncell;
    for (long c = 0; c < nc; c++) {
        double w[OMAXV], q[OMAXV];
        for (int v = 0; v < s->nvar; v++) q[v] = s->U[v * nc + c];
        cons_to_prim(s, q, w);
        for (int v = 0; v < s->nvar; v++) prim[v * nc + c] = w[v];
    }
}

void o_set_cons(void *h, const double *cons)
{
    ostate *s = (ostate *)h;
    memcpy(s->U, cons, sizeof(double) * s->nvar * s->ncell);
}

void o_get_cons(void *h, double *cons)
{
    ostate *s = (ostate *)h;
    memcpy(cons, s->U, sizeof(double) * s->nvar * s->ncell);
}

void o_set_body(void *h, const double vr[3], const double xb[3], double mass, int dynamic)
{
    ostate *s = (ostate *)h;
    for (int d = 0; d < 3; d++) {
        s->vr[d] = (d < s->dim) ? vr[d] : 0.0;
        s->xb[d] = xb[d];
    }
    s->mass = mass;
    s->dynamic = dynamic;
}

void o_get_body(void *h, double force[3], double vr[3], double xb[3])
{
    ostate *s = (ostate *)h;
    for (int d = 0; d < 3; d++) {
        force[d] = s->force[d];
        vr[d] = s->vr[d];
        xb[d] = s->xb[d];
    }
}

/* D(U) of the current state (no seeding), for tests. */
void o_compute_D(void *h, double *D)
{
    ostate *s = (ostate *)h;
    compute_D(s, s->U, D);
}

void o_seed_state(void *h) { o_seed((ostate *)h); }
void o_force_state(void *h, double F[3]) { o_force((ostate *)h, F); }
void o_plastic_state(void *h, double dt)
{
    ostate *s = (ostate *)h;
    memset(s->mask, 0, (size_t)s->ncell);
    o_plastic(s, dt);
}

/* Closure of one conserved cell vector: p, c, G, sigma_Y and J^2. */
void o_cell_closure(void *h, const double *q, double out[5])
{
    ostate *s = (ostate *)h;
    double w[OMAXV];
    othermo t;
    cons_to_prim(s, q, w);
    thermo_from_prim(s, w, &t);
    out[0] = t.p;
    out[1] = sqrt(t.c2);
    out[2] = t.G;
    out[3] = t.sigY;
    out[4] = t.J2;
}

void o_cell_prim_to_cons(void *h, const double *w, double *q) { prim_to_cons((ostate *)h, w, q); }
void o_cell_cons_to_prim(void *h, const double *q, double *w) { cons_to_prim((ostate *)h, q, w); }

/* Material reference curves of material l at (rho, J^2). */
void o_material_ref(void *h, int l, double rho, double J2, double out[6])
{
    ostate *s = (ostate *)h;
    o_mat_ref(&s->mat[l], rho, J2, out);
}

/* HLLC at one face in direction d from primitive face states. */
void o_riemann(void *h, int d, const double *wL, const double *wR, double *F, double us[3], double vrow[3])
{
    ostate *s = (ostate *)h;
    for (int v = 0; v < s->nvar; v++) F[v] = 0.0;
    o_hllc(s, d, wL, wR, F, us, vrow);
}

void o_plastic_cons(void *h, double *q, double dt) { plastic_cell((ostate *)h, q, dt); }

/* Johnson-Cook constants of material l (Table 2); c1 = c2 = 0 switches it off. */
void o_set_jc(void *h, int l, double c1, double c2, double c3, double n, double m, double tmelt, double cv)
{
    omat *mt = &((ostate *)h)->mat[l];
    mt->jc = (c1 > 0.0 || c2 > 0.0) ? 1 : 0;
    mt->jc_c1 = c1;
    mt->jc_c2 = c2;
    mt->jc_c3 = c3;
    mt->jc_n = n;
    mt->jc_m = m;
    mt->jc_tmelt = tmelt;
    mt->jc_cv = cv;
}
