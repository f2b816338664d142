// nci.cu -- batched FP64 root solver of the numerical dispersion relation of
// a relativistically drifting cold plasma on the hybrid solver's grid (the
// Appendix: Eq. 2dmodesres with the coupling term, the hybrid operators
// [k]E1 = [k]B1 = k1, [k]E2 = [k]B2 = sin(k2 dx2/2)/(dx2/2), and the cubic
// Eq. asym1 about the beam resonance).  One thread per (sample, alias): the
// cubic's roots (plus three fixed seeds around the resonance) start Newton
// iterations on F(w) = D(w) (w' - k1' v0); the largest imaginary part of the
// converged roots is the NCI growth rate of that alias, and the sample's
// growth is the largest over its aliases.
//
// Readings (the printed forms are garbled here): s_{l,i} = sinc(k'_i dx_i/2)^(l+1)
// with k' aliased; S'_B3 = S_B3; the current filter F(k1) and the j1
// correction multiply S_j1, F multiplies S_j2; momentum-conserving
// interpolation.
#include <math.h>

#include "hyb_internal.cuh"

namespace hyb {

struct Z { double re, im; };
__device__ __forceinline__ Z zc(double a, double b) { Z z; z.re = a; z.im = b; return z; }
__device__ __forceinline__ Z zadd(Z a, Z b) { return zc(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ Z zsub(Z a, Z b) { return zc(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ Z zmul(Z a, Z b) { return zc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ Z zsc(Z a, double s) { return zc(a.re * s, a.im * s); }
__device__ __forceinline__ Z zdiv(Z a, Z b) {
    // scaled division (Smith's method)
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return zc((a.re + a.im * r) / d, (a.im - a.re * r) / d);
    }
    const double r = b.re / b.im, d = b.re * r + b.im;
    return zc((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
__device__ __forceinline__ double zabs(Z a) { return hypot(a.re, a.im); }
// sin(x + iy) = sin x cosh y + i cos x sinh y
__device__ __forceinline__ Z zsin(Z a) {
    double s, c;
    sincos(a.re, &s, &c);
    return zc(s * cosh(a.im), c * sinh(a.im));
}

__device__ __forceinline__ double dsinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

struct NciMode {
    double dt, v0, a, b, k1, k2, k1a, kE1, kE2, SE1, SE2, SB3, Sj1, Sj2;
    int mu, nu1;
};

__device__ Z nci_F(const NciMode& m, Z w) {
    const double wg = 2.0 * 3.14159265358979323846 / m.dt;
    const Z wp = zc(w.re + m.mu * wg, w.im);
    const Z Delta = zc(wp.re - m.k1a * m.v0, wp.im);
    const Z wb = zsc(zsin(zsc(w, 0.5 * m.dt)), 2.0 / m.dt);
    const double K2 = m.kE1 * m.kE1 + m.kE2 * m.kE2;
    const Z first = zsub(zmul(Delta, Delta), zsc(zdiv(wp, wb), m.a * m.Sj1 * m.SE1));
    const Z second = zsub(zmul(zsub(zmul(wb, wb), zc(K2, 0.0)), Delta),
                          zsc(zsub(zsc(wb, m.SE2), zc(m.SB3 * m.kE1 * m.v0, 0.0)), m.b * m.Sj2));
    const double kE2s = m.kE2 * m.kE2;
    Z brace = zsc(wp, m.Sj1 * m.SE1 * kE2s * (m.v0 * m.v0 - 1.0));
    brace = zadd(brace, zsc(Delta, m.Sj2 * m.SE2 * kE2s));
    brace = zadd(brace, zsub(zc(m.Sj1 * m.kE2 * m.SE2 * m.kE1 * m.k2 * m.v0, 0.0), zsc(wb, m.Sj1 * m.kE2 * m.SB3 * m.k2 * m.v0 * m.v0)));
    const Z C = zsc(zdiv(brace, wb), m.b);
    return zadd(zmul(first, second), zmul(C, Delta));
}

__device__ bool nci_newton(const NciMode& m, Z w, Z* out) {
    for (int it = 0; it < 60; it++) {
        const Z f = nci_F(m, w);
        const double h = 1e-7 * fmax(1.0, zabs(w));
        const Z d = zsc(zsub(nci_F(m, zc(w.re + h, w.im)), nci_F(m, zc(w.re - h, w.im))), 0.5 / h);
        if (d.re == 0.0 && d.im == 0.0) return false;
        const Z step = zdiv(f, d);
        w = zsub(w, step);
        if (!(isfinite(w.re) && isfinite(w.im))) return false;
        if (zabs(step) <= 1e-13 * fmax(1.0, zabs(w))) { *out = w; return true; }
    }
    return false;
}

// real roots of a x^3 + b x^2 + c x + d (a != 0) and complex pair, by the companion-free closed form
__device__ int cubic_roots(double a, double b, double c, double d, Z r[3]) {
    const double A = b / a, B = c / a, C = d / a;
    const double Q = (3.0 * B - A * A) / 9.0, R = (9.0 * A * B - 27.0 * C - 2.0 * A * A * A) / 54.0;
    const double D = Q * Q * Q + R * R;
    if (D >= 0.0) {
        const double sD = sqrt(D);
        const double S = cbrt(R + sD), T = cbrt(R - sD);
        r[0] = zc(-A / 3.0 + (S + T), 0.0);
        r[1] = zc(-A / 3.0 - 0.5 * (S + T), 0.5 * sqrt(3.0) * (S - T));
        r[2] = zc(-A / 3.0 - 0.5 * (S + T), -0.5 * sqrt(3.0) * (S - T));
    } else {
        const double th = acos(R / sqrt(-Q * Q * Q));
        const double sq = 2.0 * sqrt(-Q);
        const double pi = 3.14159265358979323846;
        r[0] = zc(sq * cos(th / 3.0) - A / 3.0, 0.0);
        r[1] = zc(sq * cos((th + 2.0 * pi) / 3.0) - A / 3.0, 0.0);
        r[2] = zc(sq * cos((th + 4.0 * pi) / 3.0) - A / 3.0, 0.0);
    }
    return 3;
}

struct NciSample { double dt, dx1, dx2, gamma, wp2, filt_kc, filt_w, k1, k2; };

__device__ double filt_factor(const NciSample& s) {
    if (!(s.filt_kc > 0.0 && s.filt_kc < 1.0)) return 1.0;
    const double pi = 3.14159265358979323846, kn = pi / s.dx1, k = fabs(s.k1);
    const double kc = s.filt_kc * kn, w = s.filt_w * kn;
    if (k <= kc - 0.5 * w) return 1.0;
    if (k >= kc + 0.5 * w) return 0.0;
    const double c = cos(0.5 * pi * (k - kc + 0.5 * w) / w);
    return c * c;
}

__global__ void k_nci(const NciSample* __restrict__ smp, int64_t n, int order, int correct_j1,
                      const int* __restrict__ alias, int n_alias, double* __restrict__ growth, double2* __restrict__ root) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= n * n_alias) return;
    const int64_t i = tid / n_alias;
    const int ai = (int)(tid % n_alias);
    const NciSample s = smp[i];
    const double pi = 3.14159265358979323846;
    NciMode m;
    m.dt = s.dt;
    m.v0 = sqrt(1.0 - 1.0 / (s.gamma * s.gamma));
    m.mu = alias[2 * ai];
    m.nu1 = alias[2 * ai + 1];
    const double sgnmu = (m.mu & 1) ? -1.0 : 1.0;
    m.a = s.wp2 / (s.gamma * s.gamma * s.gamma) * sgnmu;
    m.b = s.wp2 / s.gamma * sgnmu;
    m.k1 = s.k1;
    m.k2 = s.k2;
    m.k1a = s.k1 + m.nu1 * 2.0 * pi / s.dx1;
    const double s1 = dsinc(0.5 * m.k1a * s.dx1), s2 = dsinc(0.5 * s.k2 * s.dx2);
    const double sl1 = pow(s1, order + 1), sl2 = pow(s2, order + 1), sm1 = pow(s1, order), sm2 = pow(s2, order);
    const double sgn = (m.nu1 & 1) ? -1.0 : 1.0;
    m.SE1 = sl1 * sl2 * sgn;
    m.SE2 = sl1 * sl2;
    m.SB3 = sl1 * sl2 * sgn;
    const double F = filt_factor(s);
    const double corr = (correct_j1 && s.k1 != 0.0) ? dsinc(0.5 * s.k1 * s.dx1) : 1.0;
    m.Sj1 = sm1 * sl2 * sgn * F * corr;
    m.Sj2 = sl1 * sm2 * F;
    m.kE1 = s.k1;
    m.kE2 = sin(0.5 * s.k2 * s.dx2) / (0.5 * s.dx2);
    // cubic seeds about w' = k1' v0 (Eq. asym1; v0 -> 1 inside k~1)
    const double wg = 2.0 * pi / s.dt;
    const double wres = m.k1a * m.v0 - m.mu * wg;
    const double kt = m.k1a - m.mu * wg, h = 0.5 * s.dt;
    const double xi0 = sin(kt * h) / h, xi1 = cos(kt * h), ze0 = cos(kt * h), ze1 = -sin(kt * h) * h;
    const double kE1 = m.kE1, kE2 = m.kE2;
    const double A2 = 2.0 * xi0 * xi0 * xi0 * xi1;
    const double B2 = xi0 * xi0 * (xi0 * xi0 - kE1 * kE1 - kE2 * kE2 - m.b * m.Sj2 * (m.SE2 * xi1 - ze1 * m.SB3 * kE1));
    const double C2 = m.b * (xi0 * xi0 * m.Sj2 * (ze0 * m.SB3 * kE1 - m.SE2 * xi0) - xi1 * m.Sj1 * kE2 * m.k2 * m.SE2 * kE1
                             + xi0 * kE2 * (m.Sj2 * m.SE2 * kE2 - m.Sj1 * m.k2 * ze1 * m.SB3 * xi0));
    const double D2 = m.b * xi0 * kE2 * m.k2 * m.Sj1 * (m.SE2 * kE1 - ze0 * m.SB3 * xi0);
    Z seeds[6];
    int ns = 0;
    if (A2 != 0.0) {
        Z r[3];
        cubic_roots(A2, B2, C2, D2, r);
        for (int q = 0; q < 3; q++) seeds[ns++] = zc(wres + r[q].re, r[q].im);
    }
    const double r0 = cbrt(s.wp2 / s.gamma) * 0.05;
    const double th[3] = {pi / 6.0, pi / 2.0, 5.0 * pi / 6.0};
    for (int q = 0; q < 3; q++) seeds[ns++] = zc(wres + r0 * cos(th[q]), r0 * sin(th[q]));
    double best = 0.0;
    Z broot = zc(wres, 0.0);
    for (int q = 0; q < ns; q++) {
        Z w;
        if (!nci_newton(m, seeds[q], &w)) continue;
        const double dres = hypot(w.re + m.mu * wg - m.k1a * m.v0, w.im);
        if (dres < 1e-9 * fmax(1.0, zabs(w))) continue;       // the removed resonance pole
        if (w.im > best) { best = w.im; broot = w; }
    }
    growth[tid] = best;
    if (root) root[tid] = make_double2(broot.re, broot.im);
}

}  // namespace hyb

using namespace hyb;

extern "C" hyb_status hyb_nci_growth(const double* samples, int64_t n, int order, int correct_j1,
                                     const int* alias, int n_alias, double* growth, double* root, void* stream) {
    if (!samples || !alias || !growth || n < 0 || n_alias < 1 || order < 1 || order > 3) {
        set_error("hyb_nci_growth: bad arguments");
        return HYB_EINVAL;
    }
    if (n == 0) return HYB_OK;
    const int64_t total = n * n_alias;
    const int thr = 128;
    k_nci<<<(unsigned)((total + thr - 1) / thr), thr, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const NciSample*>(samples), n, order, correct_j1, alias, n_alias, growth,
        reinterpret_cast<double2*>(root));
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}
