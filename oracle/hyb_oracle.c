/*
 * hyb_oracle.c -- plain, slow, FP64 CPU oracle of the hybrid Yee-FFT field
 * advance (Yu et al., "Mitigation of numerical Cerenkov radiation and
 * instability using a hybrid finite difference-FFT Maxwell solver and a local
 * charge conserving current deposit", arXiv:1502.01376).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it has its own textbook FFT.
 *
 * Conventions (the reading every function below follows):
 *   - arrays are row-major [n3][n2][n1] (n3 = 1 in 2D), x1 contiguous;
 *   - a half-integer position i+1/2 is stored at index i (Yee staggering of
 *     Sec. 2.1: E1(i1+1/2,i2), E2(i1,i2+1/2), E3(i1,i2), B1(i1,i2+1/2),
 *     B2(i1+1/2,i2), B3(i1+1/2,i2+1/2), j like E, rho at (i1,i2); in 3D the
 *     standard Yee cell: E3 at k+1/2, B1 at (j+1/2,k+1/2), B2 at (i+1/2,k+1/2));
 *   - forward DFT along x1: F[kappa] = sum_j f[j] exp(-2 pi i kappa j / n1),
 *     k1 = 2 pi kappa / (n1 dx1), kappa = 0..n1/2 kept (Nyquist included);
 *   - the hybrid x1 derivative from integer to half-integer points has symbol
 *     sigma+ = i [k]1 exp(+i k1 dx1/2), from half-integer to integer points
 *     sigma- = i [k]1 exp(-i k1 dx1/2), where [k]1 = k1 for the hybrid solver
 *     (Sec. 2.1, "replace [k]1 by k1"), [k]1 = sin(k1 dx1/2)/(dx1/2) for the
 *     Yee-recovery mode (Sec. 2.1, last sentence), and [k]1 = k1 + dk_mod(k1)
 *     inside the dispersion bump of Sec. 4;
 *   - c = 1 (normalised units, Table 1); Ampere coefficient 4 pi (Eq. yee2de1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int dims;                 /* 2 or 3 */
    int n1, n2, n3;           /* grid points; n3 ignored (=1) in 2D */
    double dx1, dx2, dx3, dt;
    int correct_j1;           /* Eq. currentcorrection on/off */
    double filt_kc, filt_w;   /* low-pass filter of Sec. 4, fractions of pi/dx1; on iff 0<kc<1 */
    double kmod_l, kmod_u, kmod_max; /* dispersion bump of Sec. 4, fractions of k_g1=2pi/dx1 */
    int yee_mode;             /* [k]1 = sin(k1 dx1/2)/(dx1/2) instead of k1 */
    double ampere;            /* coefficient of j in Ampere's law (4 pi) */
} orc_grid;

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx csub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static inline cplx cscale(cplx a, double s) { cplx r = {a.re * s, a.im * s}; return r; }

/* ------------------------------------------------------------------------ */
/* Textbook FFT: iterative radix-2 Cooley-Tukey for powers of two, a direct  */
/* O(n^2) DFT otherwise.  sign = -1: forward, +1: inverse (unnormalised).     */
/* ------------------------------------------------------------------------ */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void dft_direct(cplx* z, int n, int sign) {
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int k = 0; k < n; k++) {
        cplx s = {0.0, 0.0};
        for (int j = 0; j < n; j++) {
            long long m = ((long long)j * k) % n;
            double ang = sign * 2.0 * ORC_PI * (double)m / (double)n;
            cplx w = {cos(ang), sin(ang)};
            s = cadd(s, cmul(z[j], w));
        }
        out[k] = s;
    }
    memcpy(z, out, sizeof(cplx) * (size_t)n);
    free(out);
}

static void fft_radix2(cplx* z, int n, int sign) {
    for (int i = 1, j = 0; i < n; i++) {           /* bit-reversal permutation */
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = z[i]; z[i] = z[j]; z[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {       /* butterflies of span len */
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            double ang = sign * 2.0 * ORC_PI * (double)k / (double)len;
            cplx w = {cos(ang), sin(ang)};
            for (int i = 0; i < n; i += len) {
                cplx u = z[i + k];
                cplx v = cmul(z[i + k + half], w);
                z[i + k] = cadd(u, v);
                z[i + k + half] = csub(u, v);
            }
        }
    }
}

void orc_fft(double* zi, int n, int sign) {
    cplx* z = (cplx*)zi;
    if (is_pow2(n)) fft_radix2(z, n, sign); else dft_direct(z, n, sign);
}

/* real line -> kappa = 0..n/2 (n even), via a full complex transform */
static void rfft_line(const double* x, int n, cplx* X, cplx* work) {
    for (int j = 0; j < n; j++) { work[j].re = x[j]; work[j].im = 0.0; }
    orc_fft((double*)work, n, -1);
    for (int k = 0; k <= n / 2; k++) X[k] = work[k];
}

/* kappa = 0..n/2 -> real line; Hermitian extension, imaginary parts of the
 * DC and Nyquist bins dropped, normalised by 1/n. */
static void irfft_line(const cplx* X, int n, double* x, cplx* work) {
    for (int k = 0; k <= n / 2; k++) work[k] = X[k];
    work[0].im = 0.0;
    work[n / 2].im = 0.0;
    for (int k = 1; k < n / 2; k++) { work[n - k].re = X[k].re; work[n - k].im = -X[k].im; }
    orc_fft((double*)work, n, +1);
    for (int j = 0; j < n; j++) x[j] = work[j].re / (double)n;
}

void orc_rfft(const double* x, int n, double* X) {
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    rfft_line(x, n, (cplx*)X, w);
    free(w);
}

void orc_irfft(const double* X, int n, double* x) {
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    irfft_line((const cplx*)X, n, x, w);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Per-mode tables (kappa = 0..n1/2)                                          */
/* ------------------------------------------------------------------------ */
static double k1_of(const orc_grid* g, int kappa) { return 2.0 * ORC_PI * kappa / (g->n1 * g->dx1); }

/* finite-difference symbol [k]1 = sin(k1 dx1/2)/(dx1/2) (Sec. 2.1) */
static double kfd_of(const orc_grid* g, int kappa) {
    double k = k1_of(g, kappa);
    return sin(0.5 * k * g->dx1) / (0.5 * g->dx1);
}

/* the x1 operator's [k]1: k1 (hybrid), [k]1 FD (Yee recovery), or with the
 * Sec. 4 bump dk_mod = dk_max cos^2(pi/2 (k1-k1m)/(k1l-k1m)) on [k1l,k1u]. */
static double keff_of(const orc_grid* g, int kappa) {
    if (g->yee_mode) return kfd_of(g, kappa);
    double k = k1_of(g, kappa);
    if (g->kmod_max != 0.0) {
        double kg = 2.0 * ORC_PI / g->dx1;
        double kl = g->kmod_l * kg, ku = g->kmod_u * kg, km = 0.5 * (kl + ku);
        if (k >= kl && k <= ku) {
            double c = cos(0.5 * ORC_PI * (k - km) / (kl - km));
            k += g->kmod_max * kg * c * c;
        }
    }
    return k;
}

/* Eq. currentcorrection: j1 <- sin(k1dx1/2)/(k1dx1/2) j1.  Written as
 * [k]1_FD / [k]1 so that it is 1 in the Yee-recovery mode and keeps the
 * continuity equation consistent with the bump (reading of Sec. 4). */
static double corr_of(const orc_grid* g, int kappa) {
    if (kappa == 0) return 1.0;
    return kfd_of(g, kappa) / keff_of(g, kappa);
}

/* Sec. 4 low-pass "form factor" on the current in k1: raised cosine,
 * 1 below kc-w/2, cos^2 across the transition, 0 above kc+w/2 (F(kc) = 1/2). */
static double filt_of(const orc_grid* g, int kappa) {
    if (!(g->filt_kc > 0.0 && g->filt_kc < 1.0)) return 1.0;
    double kn = ORC_PI / g->dx1;
    double k = fabs(k1_of(g, kappa));
    double kc = g->filt_kc * kn, w = g->filt_w * kn;
    if (w <= 0.0) return k <= kc ? 1.0 : 0.0;
    if (k <= kc - 0.5 * w) return 1.0;
    if (k >= kc + 0.5 * w) return 0.0;
    double c = cos(0.5 * ORC_PI * (k - kc + 0.5 * w) / w);
    return c * c;
}

void orc_mode_tables(const orc_grid* g, double* keff, double* corr, double* filt) {
    for (int k = 0; k <= g->n1 / 2; k++) {
        if (keff) keff[k] = keff_of(g, k);
        if (corr) corr[k] = corr_of(g, k);
        if (filt) filt[k] = filt_of(g, k);
    }
}

/* Courant limit of Sec. 2.2: dt <= 2 / sqrt(pi^2/dx1^2 + 4/dx2^2 [+ 4/dx3^2]) */
double orc_courant(const orc_grid* g) {
    double s = ORC_PI * ORC_PI / (g->dx1 * g->dx1) + 4.0 / (g->dx2 * g->dx2);
    if (g->dims == 3) s += 4.0 / (g->dx3 * g->dx3);
    return 2.0 / sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Spectral field arrays                                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int n1, nk, n2, n3; size_t rows; } shape_t;

static shape_t shape_of(const orc_grid* g) {
    shape_t s;
    s.n1 = g->n1; s.nk = g->n1 / 2 + 1; s.n2 = g->n2; s.n3 = (g->dims == 3) ? g->n3 : 1;
    s.rows = (size_t)s.n2 * s.n3;
    return s;
}

static void forward_all(const shape_t* s, const double* f, cplx* F) {
    #pragma omp parallel
    {
        cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)s->n1);
        #pragma omp for schedule(static)
        for (long r = 0; r < (long)s->rows; r++) rfft_line(f + (size_t)r * s->n1, s->n1, F + (size_t)r * s->nk, w);
        free(w);
    }
}

static void inverse_all(const shape_t* s, const cplx* F, double* f) {
    #pragma omp parallel
    {
        cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)s->n1);
        #pragma omp for schedule(static)
        for (long r = 0; r < (long)s->rows; r++) irfft_line(F + (size_t)r * s->nk, s->n1, f + (size_t)r * s->n1, w);
        free(w);
    }
}

/* sigma+/- = i [k]1 exp(+/- i k1 dx1/2) */
static void sigma_tables(const orc_grid* g, cplx* sp, cplx* sm) {
    for (int k = 0; k <= g->n1 / 2; k++) {
        double ke = keff_of(g, k), ph = 0.5 * k1_of(g, k) * g->dx1;
        cplx ik = {0.0, ke};
        cplx ep = {cos(ph), sin(ph)}, em = {cos(ph), -sin(ph)};
        sp[k] = cmul(ik, ep);
        sm[k] = cmul(ik, em);
    }
}

/* ------------------------------------------------------------------------ */
/* One or more steps of the hybrid advance (Eqs. hybrid2db1-hybrid2de3; the   */
/* 3D form of Sec. 2.4 adds the x3 Yee differences).                          */
/* On entry E = E^n, B = B^{n-1/2}, J = j^{n+1/2}; on exit E^{n+1}, B^{n+1/2}. */
/* The same J is used for every one of the nsteps steps.                      */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_grid* g, double* E1, double* E2, double* E3,
             double* B1, double* B2, double* B3,
             const double* J1, const double* J2, const double* J3, int nsteps) {
    if (g->n1 < 2 || (g->n1 & 1) || g->n2 < 1) return -1;
    shape_t s = shape_of(g);
    size_t ncx = s.rows * (size_t)s.nk;
    double* Er[3] = {E1, E2, E3};
    double* Br[3] = {B1, B2, B3};
    const double* Jr[3] = {J1, J2, J3};
    cplx* buf = (cplx*)malloc(sizeof(cplx) * ncx * 9);
    if (!buf) return -2;
    cplx *Eh[3], *Bh[3], *Jh[3];
    for (int c = 0; c < 3; c++) { Eh[c] = buf + c * ncx; Bh[c] = buf + (3 + c) * ncx; Jh[c] = buf + (6 + c) * ncx; }
    cplx* sp = (cplx*)malloc(sizeof(cplx) * s.nk);
    cplx* sm = (cplx*)malloc(sizeof(cplx) * s.nk);
    double* corr = (double*)malloc(sizeof(double) * s.nk);
    double* filt = (double*)malloc(sizeof(double) * s.nk);
    sigma_tables(g, sp, sm);
    orc_mode_tables(g, NULL, corr, filt);

    const double a = g->dt;                  /* c dt, c = 1 */
    const double a2 = g->dt / g->dx2;
    const double a3 = (g->dims == 3) ? g->dt / g->dx3 : 0.0;
    const double aj = g->ampere * g->dt;
    const int d3 = (g->dims == 3);
    const int n2 = s.n2, n3 = s.n3, nk = s.nk;

    for (int step = 0; step < nsteps; step++) {
        for (int c = 0; c < 3; c++) {
            forward_all(&s, Er[c], Eh[c]);
            forward_all(&s, Br[c], Bh[c]);
            forward_all(&s, Jr[c], Jh[c]);
        }
        /* current correction (Eq. currentcorrection) and k1 filter (Sec. 4) */
        for (size_t r = 0; r < s.rows; r++)
            for (int k = 0; k < nk; k++) {
                size_t i = r * nk + k;
                double f1 = filt[k] * (g->correct_j1 ? corr[k] : 1.0);
                Jh[0][i] = cscale(Jh[0][i], f1);
                Jh[1][i] = cscale(Jh[1][i], filt[k]);
                Jh[2][i] = cscale(Jh[2][i], filt[k]);
            }
        /* Faraday: B^{n+1/2} from E^n, all rows */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int i3 = 0; i3 < n3; i3++)
            for (int i2 = 0; i2 < n2; i2++) {
                size_t r = (size_t)i3 * n2 + i2;
                size_t rp2 = (size_t)i3 * n2 + (i2 + 1) % n2;           /* i2+1 */
                size_t rp3 = (size_t)((i3 + 1) % n3) * n2 + i2;         /* i3+1 */
                for (int k = 0; k < nk; k++) {
                    size_t i = r * nk + k, ip2 = rp2 * nk + k, ip3 = rp3 * nk + k;
                    cplx e1 = Eh[0][i], e2 = Eh[1][i], e3 = Eh[2][i];
                    cplx d2e3 = cscale(csub(Eh[2][ip2], e3), a2);
                    cplx d2e1 = cscale(csub(Eh[0][ip2], e1), a2);
                    cplx d3e2 = {0, 0}, d3e1 = {0, 0};
                    if (d3) { d3e2 = cscale(csub(Eh[1][ip3], e2), a3); d3e1 = cscale(csub(Eh[0][ip3], e1), a3); }
                    cplx d1e3 = cscale(cmul(sp[k], e3), a);
                    cplx d1e2 = cscale(cmul(sp[k], e2), a);
                    /* B1 -= c dt (d2 E3 - d3 E2) */
                    Bh[0][i] = csub(Bh[0][i], csub(d2e3, d3e2));
                    /* B2 -= c dt (d3 E1 - d1 E3) */
                    Bh[1][i] = csub(Bh[1][i], csub(d3e1, d1e3));
                    /* B3 -= c dt (d1 E2 - d2 E1) */
                    Bh[2][i] = csub(Bh[2][i], csub(d1e2, d2e1));
                }
            }
        /* Ampere: E^{n+1} from B^{n+1/2} and the processed current */
        #pragma omp parallel for collapse(2) schedule(static)
        for (int i3 = 0; i3 < n3; i3++)
            for (int i2 = 0; i2 < n2; i2++) {
                size_t r = (size_t)i3 * n2 + i2;
                size_t rm2 = (size_t)i3 * n2 + (i2 + n2 - 1) % n2;      /* i2-1 */
                size_t rm3 = (size_t)((i3 + n3 - 1) % n3) * n2 + i2;    /* i3-1 */
                for (int k = 0; k < nk; k++) {
                    size_t i = r * nk + k, im2 = rm2 * nk + k, im3 = rm3 * nk + k;
                    cplx b1 = Bh[0][i], b2 = Bh[1][i], b3 = Bh[2][i];
                    cplx d2b3 = cscale(csub(b3, Bh[2][im2]), a2);
                    cplx d2b1 = cscale(csub(b1, Bh[0][im2]), a2);
                    cplx d3b2 = {0, 0}, d3b1 = {0, 0};
                    if (d3) { d3b2 = cscale(csub(b2, Bh[1][im3]), a3); d3b1 = cscale(csub(b1, Bh[0][im3]), a3); }
                    cplx d1b3 = cscale(cmul(sm[k], b3), a);
                    cplx d1b2 = cscale(cmul(sm[k], b2), a);
                    /* E1 += c dt (d2 B3 - d3 B2) - 4 pi dt j1~ */
                    Eh[0][i] = csub(cadd(Eh[0][i], csub(d2b3, d3b2)), cscale(Jh[0][i], aj));
                    /* E2 += c dt (d3 B1 - d1 B3) - 4 pi dt j2 */
                    Eh[1][i] = csub(cadd(Eh[1][i], csub(d3b1, d1b3)), cscale(Jh[1][i], aj));
                    /* E3 += c dt (d1 B2 - d2 B1) - 4 pi dt j3 */
                    Eh[2][i] = csub(cadd(Eh[2][i], csub(d1b2, d2b1)), cscale(Jh[2][i], aj));
                }
            }
        for (int c = 0; c < 3; c++) {
            inverse_all(&s, Eh[c], Er[c]);
            inverse_all(&s, Bh[c], Br[c]);
        }
    }
    free(buf); free(sp); free(sm); free(corr); free(filt);
    return 0;
}

/* Apply the k1-space current processing alone (correction of J1 and/or the
 * filter of all components), in place, as a standalone operation. */
int orc_process_current(const orc_grid* g, double* J1, double* J2, double* J3, int do_corr, int do_filt) {
    shape_t s = shape_of(g);
    size_t ncx = s.rows * (size_t)s.nk;
    cplx* F = (cplx*)malloc(sizeof(cplx) * ncx);
    double* corr = (double*)malloc(sizeof(double) * s.nk);
    double* filt = (double*)malloc(sizeof(double) * s.nk);
    orc_mode_tables(g, NULL, corr, filt);
    double* J[3] = {J1, J2, J3};
    for (int c = 0; c < 3; c++) {
        if (!J[c]) continue;
        if (!do_filt && !(do_corr && c == 0)) continue;
        forward_all(&s, J[c], F);
        for (size_t r = 0; r < s.rows; r++)
            for (int k = 0; k < s.nk; k++) {
                double f = (do_filt ? filt[k] : 1.0) * ((do_corr && c == 0) ? corr[k] : 1.0);
                F[r * s.nk + k] = cscale(F[r * s.nk + k], f);
            }
        inverse_all(&s, F, J[c]);
    }
    free(F); free(corr); free(filt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Particle shapes (B-splines of order l in cell units, centred on the grid   */
/* point) and the charge-conserving deposit in Esirkepov's form, which        */
/* satisfies the finite-difference continuity equation of Sec. 2.3 exactly.   */
/* ------------------------------------------------------------------------ */
double orc_shape(int order, double d) {
    double a = fabs(d);
    switch (order) {
    case 1: return a < 1.0 ? 1.0 - a : 0.0;
    case 2:
        if (a <= 0.5) return 0.75 - a * a;
        if (a < 1.5) { double t = 1.5 - a; return 0.5 * t * t; }
        return 0.0;
    case 3:
        if (a <= 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
        if (a < 2.0) { double t = 2.0 - a; return t * t * t / 6.0; }
        return 0.0;
    default: return 0.0;
    }
}

#define ORC_W 8           /* window of grid points around the start cell */
#define ORC_W0 3          /* window starts 3 points below the start cell */

static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Zeroes J and deposits j^{n+1/2} of particles moving from cell+off_old to
 * cell+off_new (positions in cell units, |off_new-off_old| < 1 per axis).
 * 2D: cell/off are [np][2], v3 gives the out-of-plane velocity for j3.
 * 3D: cell/off are [np][3], v3 unused.  Periodic in every direction. */
int orc_deposit(const orc_grid* g, const int32_t* cell, const double* off_old, const double* off_new,
                const double* v3, const double* q, int64_t np, int order,
                double* J1, double* J2, double* J3) {
    int d = g->dims;
    int n1 = g->n1, n2 = g->n2, n3 = (d == 3) ? g->n3 : 1;
    size_t nc = (size_t)n1 * n2 * n3;
    memset(J1, 0, nc * sizeof(double));
    memset(J2, 0, nc * sizeof(double));
    memset(J3, 0, nc * sizeof(double));
    double dV = g->dx1 * g->dx2 * (d == 3 ? g->dx3 : 1.0);
    for (int64_t p = 0; p < np; p++) {
        double S0[3][ORC_W], S1[3][ORC_W], dS[3][ORC_W];
        int base[3] = {0, 0, 0};
        for (int a = 0; a < d; a++) {
            base[a] = cell[p * d + a] - ORC_W0;
            for (int w = 0; w < ORC_W; w++) {
                double xi = (double)(w - ORC_W0);          /* grid point relative to the cell */
                S0[a][w] = orc_shape(order, off_old[p * d + a] - xi);
                S1[a][w] = orc_shape(order, off_new[p * d + a] - xi);
                dS[a][w] = S1[a][w] - S0[a][w];
            }
        }
        double qp = q[p];
        if (d == 2) {
            double c1 = -qp / (g->dt * g->dx2), c2 = -qp / (g->dt * g->dx1);
            double c3 = (v3 ? qp * v3[p] : 0.0) / dV;
            for (int j = 0; j < ORC_W; j++) {          /* j1: cumulative sum along x1 */
                double acc = 0.0;
                int jj = wrap(base[1] + j, n2);
                for (int i = 0; i < ORC_W; i++) {
                    acc += dS[0][i] * 0.5 * (S0[1][j] + S1[1][j]);
                    J1[(size_t)jj * n1 + wrap(base[0] + i, n1)] += c1 * acc;
                }
            }
            for (int i = 0; i < ORC_W; i++) {          /* j2: cumulative sum along x2 */
                double acc = 0.0;
                int ii = wrap(base[0] + i, n1);
                for (int j = 0; j < ORC_W; j++) {
                    acc += dS[1][j] * 0.5 * (S0[0][i] + S1[0][i]);
                    J2[(size_t)wrap(base[1] + j, n2) * n1 + ii] += c2 * acc;
                }
            }
            if (c3 != 0.0)
                for (int j = 0; j < ORC_W; j++)
                    for (int i = 0; i < ORC_W; i++) {
                        double w3 = S0[0][i] * S0[1][j] / 3.0 + S1[0][i] * S0[1][j] / 6.0
                                  + S0[0][i] * S1[1][j] / 6.0 + S1[0][i] * S1[1][j] / 3.0;
                        J3[(size_t)wrap(base[1] + j, n2) * n1 + wrap(base[0] + i, n1)] += c3 * w3;
                    }
        } else {
            double c1 = -qp / (g->dt * g->dx2 * g->dx3);
            double c2 = -qp / (g->dt * g->dx1 * g->dx3);
            double c3 = -qp / (g->dt * g->dx1 * g->dx2);
            for (int k = 0; k < ORC_W; k++)
                for (int j = 0; j < ORC_W; j++) {
                    double acc = 0.0;
                    size_t row = ((size_t)wrap(base[2] + k, n3) * n2 + wrap(base[1] + j, n2)) * n1;
                    for (int i = 0; i < ORC_W; i++) {
                        double w = dS[0][i] * (S0[1][j] * S0[2][k] + 0.5 * dS[1][j] * S0[2][k]
                                               + 0.5 * S0[1][j] * dS[2][k] + dS[1][j] * dS[2][k] / 3.0);
                        acc += w;
                        J1[row + wrap(base[0] + i, n1)] += c1 * acc;
                    }
                }
            for (int k = 0; k < ORC_W; k++)
                for (int i = 0; i < ORC_W; i++) {
                    double acc = 0.0;
                    for (int j = 0; j < ORC_W; j++) {
                        double w = dS[1][j] * (S0[0][i] * S0[2][k] + 0.5 * dS[0][i] * S0[2][k]
                                               + 0.5 * S0[0][i] * dS[2][k] + dS[0][i] * dS[2][k] / 3.0);
                        acc += w;
                        J2[((size_t)wrap(base[2] + k, n3) * n2 + wrap(base[1] + j, n2)) * n1 + wrap(base[0] + i, n1)] += c2 * acc;
                    }
                }
            for (int j = 0; j < ORC_W; j++)
                for (int i = 0; i < ORC_W; i++) {
                    double acc = 0.0;
                    for (int k = 0; k < ORC_W; k++) {
                        double w = dS[2][k] * (S0[0][i] * S0[1][j] + 0.5 * dS[0][i] * S0[1][j]
                                               + 0.5 * S0[0][i] * dS[1][j] + dS[0][i] * dS[1][j] / 3.0);
                        acc += w;
                        J3[((size_t)wrap(base[2] + k, n3) * n2 + wrap(base[1] + j, n2)) * n1 + wrap(base[0] + i, n1)] += c3 * acc;
                    }
                }
        }
    }
    return 0;
}

/* charge density rho = q S / dV at the integer grid points */
int orc_charge(const orc_grid* g, const int32_t* cell, const double* off, const double* q,
               int64_t np, int order, double* rho) {
    int d = g->dims;
    int n1 = g->n1, n2 = g->n2, n3 = (d == 3) ? g->n3 : 1;
    memset(rho, 0, (size_t)n1 * n2 * n3 * sizeof(double));
    double dV = g->dx1 * g->dx2 * (d == 3 ? g->dx3 : 1.0);
    for (int64_t p = 0; p < np; p++) {
        double S[3][ORC_W];
        int base[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++) for (int w = 0; w < ORC_W; w++) S[a][w] = (a < d) ? 0.0 : (w == 0);
        for (int a = 0; a < d; a++) {
            base[a] = cell[p * d + a] - ORC_W0;
            for (int w = 0; w < ORC_W; w++) S[a][w] = orc_shape(order, off[p * d + a] - (double)(w - ORC_W0));
        }
        int nw3 = (d == 3) ? ORC_W : 1;
        for (int k = 0; k < nw3; k++)
            for (int j = 0; j < ORC_W; j++)
                for (int i = 0; i < ORC_W; i++) {
                    double w = S[0][i] * S[1][j] * S[2][k];
                    if (w == 0.0) continue;
                    size_t idx = ((size_t)wrap(base[2] + k, n3) * n2 + wrap(base[1] + j, n2)) * n1 + wrap(base[0] + i, n1);
                    rho[idx] += q[p] * w / dV;
                }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */
/* real-space result of the hybrid x1 derivative: dir=+1 integer -> half
 * points (sigma+), dir=-1 half -> integer points (sigma-) */
static void d1_real(const orc_grid* g, const double* f, int dir, double* out) {
    shape_t s = shape_of(g);
    cplx* F = (cplx*)malloc(sizeof(cplx) * s.rows * s.nk);
    cplx* sp = (cplx*)malloc(sizeof(cplx) * s.nk);
    cplx* sm = (cplx*)malloc(sizeof(cplx) * s.nk);
    sigma_tables(g, sp, sm);
    forward_all(&s, f, F);
    for (size_t r = 0; r < s.rows; r++)
        for (int k = 0; k < s.nk; k++) F[r * s.nk + k] = cmul(dir > 0 ? sp[k] : sm[k], F[r * s.nk + k]);
    inverse_all(&s, F, out);
    free(F); free(sp); free(sm);
}

/* div B at (i1+1/2, i2+1/2[, i3+1/2]) = sigma+ B1 + d2+ B2 [+ d3+ B3] */
int orc_divb(const orc_grid* g, const double* B1, const double* B2, const double* B3, double* out) {
    shape_t s = shape_of(g);
    d1_real(g, B1, +1, out);
    for (int i3 = 0; i3 < s.n3; i3++)
        for (int i2 = 0; i2 < s.n2; i2++)
            for (int i1 = 0; i1 < s.n1; i1++) {
                size_t i = ((size_t)i3 * s.n2 + i2) * s.n1 + i1;
                size_t ip2 = ((size_t)i3 * s.n2 + (i2 + 1) % s.n2) * s.n1 + i1;
                out[i] += (B2[ip2] - B2[i]) / g->dx2;
                if (g->dims == 3) {
                    size_t ip3 = ((size_t)((i3 + 1) % s.n3) * s.n2 + i2) * s.n1 + i1;
                    out[i] += (B3[ip3] - B3[i]) / g->dx3;
                }
            }
    return 0;
}

/* Gauss residual at the integer points (Sec. 2.3):
 * sigma- E1 + d2- E2 [+ d3- E3] - 4 pi F rho, with F the k1 filter of the
 * current (the quantity whose time derivative vanishes when the corrected and
 * filtered current drives Ampere's law).  rho may be NULL (treated as 0). */
int orc_gauss(const orc_grid* g, const double* E1, const double* E2, const double* E3,
              const double* rho, double* out) {
    shape_t s = shape_of(g);
    size_t nc = s.rows * (size_t)s.n1;
    d1_real(g, E1, -1, out);
    for (int i3 = 0; i3 < s.n3; i3++)
        for (int i2 = 0; i2 < s.n2; i2++)
            for (int i1 = 0; i1 < s.n1; i1++) {
                size_t i = ((size_t)i3 * s.n2 + i2) * s.n1 + i1;
                size_t im2 = ((size_t)i3 * s.n2 + (i2 + s.n2 - 1) % s.n2) * s.n1 + i1;
                out[i] += (E2[i] - E2[im2]) / g->dx2;
                if (g->dims == 3) {
                    size_t im3 = ((size_t)((i3 + s.n3 - 1) % s.n3) * s.n2 + i2) * s.n1 + i1;
                    out[i] += (E3[i] - E3[im3]) / g->dx3;
                }
            }
    if (rho) {
        double* fr = (double*)malloc(sizeof(double) * nc);
        memcpy(fr, rho, sizeof(double) * nc);
        orc_process_current(g, fr, NULL, NULL, 0, 1);   /* F rho */
        for (size_t i = 0; i < nc; i++) out[i] -= g->ampere * fr[i];
        free(fr);
    }
    return 0;
}

/* out[0..5]: sum f^2 dV / (8 pi) for E1,E2,E3,B1,B2,B3; out[6]: max |div B|;
 * out[7]: max |Gauss residual|; out[8]: rms Gauss residual. */
int orc_diag(const orc_grid* g, const double* E1, const double* E2, const double* E3,
             const double* B1, const double* B2, const double* B3, const double* rho, double* out) {
    shape_t s = shape_of(g);
    size_t nc = s.rows * (size_t)s.n1;
    double dV = g->dx1 * g->dx2 * (g->dims == 3 ? g->dx3 : 1.0);
    const double* f[6] = {E1, E2, E3, B1, B2, B3};
    for (int c = 0; c < 6; c++) {
        double acc = 0.0;
        for (size_t i = 0; i < nc; i++) acc += f[c][i] * f[c][i];
        out[c] = acc * dV / (8.0 * ORC_PI);
    }
    double* w = (double*)malloc(sizeof(double) * nc);
    orc_divb(g, B1, B2, B3, w);
    double m = 0.0;
    for (size_t i = 0; i < nc; i++) m = fmax(m, fabs(w[i]));
    out[6] = m;
    orc_gauss(g, E1, E2, E3, rho, w);
    m = 0.0;
    double ss = 0.0;
    for (size_t i = 0; i < nc; i++) { m = fmax(m, fabs(w[i])); ss += w[i] * w[i]; }
    out[7] = m;
    out[8] = sqrt(ss / (double)nc);
    free(w);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
