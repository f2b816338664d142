// nci.cu -- batched FP64 root solver of the numerical dispersion relation of
// a relativistically drifting cold plasma on the hybrid solver's grid (the
// Appendix: Eq. 2dmodesres with the coupling term, the hybrid operators
// [k]E1 = [k]B1 = k1 (plus the Sec. 4 bump), [k]E2 = [k]B2 =
// sin(k2 dx2/2)/(dx2/2), and the cubic Eq. asym1 about the beam resonance).
//
// One thread per (sample, alias).  The roots sought are all zeros of
//   G(w) = [w] D(w) (w' - k1' v0)
// (the relation times the factors that remove its poles: G is entire) in the
// disk |w - w_res| < rho about the beam resonance w' = k1' v0, with
// rho = (wp2/gamma)^(1/3), the scale at which the cubic's leading and
// constant terms balance.  The growth rate of the alias is the largest Im w
// over them (0 if none grows); a sample's growth is the largest over its
// aliases.
//
//  1. The number N of zeros in the disk: the winding of G along the circle
//     (phase steps sampled until none exceeds 0.5 rad).
//  2. Newton's method with G' from the product rule, deflated by the zeros
//     already found (step 1 / (G'/G - sum 1/(w - r_j)), so no zero is found
//     twice), from seeds: the cubic's roots, the resonance itself and rings
//     inside the disk; done when N zeros inside the disk are found.
//  3. If the seeds leave zeros unfound, the rectangle around the disk is split
//     into four pieces whose zeros are counted by their boundary's winding,
//     recursively, and Newton's method is run inside each piece that holds
//     one zero (complete by construction).
//
// Readings (the printed forms are garbled here): s_{l,i} = sinc(k'_i dx_i/2)^(l+1)
// with k' aliased; S_B3 = S'_B3 cos(w dt/2), B's time centring, whose
// expansion about the resonance is the cubic's zeta0 + zeta1 dw'; the current
// filter F(k1) and the j1 correction multiply S_j1, F multiplies S_j2;
// momentum-conserving interpolation.
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

__device__ __forceinline__ double dsinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

// The symbols of one (sample, alias).
struct NciMode {
    double h, v0, a, b, wg, k1a, kE1, kE2, k2, SE1, SE2, SB3s, Sj1, Sj2;
    int mu;
};

// G(w) and G'(w).  With u = w h (h = dt/2): [w] = sin(u)/h, c = cos(u) (B's time
// centring), d[w]/dw = c, dc/dw = -h sin(u) = -h^2 [w].
//   A = [w] (Delta^2) - a Sj1 SE1 w'                                 ([w] x first factor)
//   S = ([w]^2 - K2) Delta - b Sj2 (SE2 [w] - SB3 kE1 v0)             (second factor x Delta)
//   C = b (Sj1 SE1 w' kE2^2 (v0^2 - 1) + Sj2 SE2 kE2^2 Delta
//          + Sj1 kE2 k2 (SE2 kE1 v0 - SB3 v0^2 [w]))                  ([w] x coupling term)
//   G = A S + C Delta,  SB3 = SB3s c.
__device__ void nci_G(const NciMode& m, Z w, Z* g, Z* dg) {
    double su, cu;
    sincos(w.re * m.h, &su, &cu);
    const double ch = cosh(w.im * m.h), sh = sinh(w.im * m.h);
    const Z sn = zc(su * ch, cu * sh);                  // sin(w h)
    const Z cs = zc(cu * ch, -su * sh);                 // cos(w h)
    const Z wb = zsc(sn, 1.0 / m.h);
    const Z dwb = cs;
    const Z dcs = zsc(sn, -m.h);
    const Z wp = zc(w.re + m.mu * m.wg, w.im);
    const Z D = zc(wp.re - m.k1a * m.v0, wp.im);        // Delta; dDelta/dw = 1, dw'/dw = 1
    const double K2 = m.kE1 * m.kE1 + m.kE2 * m.kE2, kE2s = m.kE2 * m.kE2;
    const Z D2 = zmul(D, D);
    // A and A'
    const Z A = zsub(zmul(wb, D2), zsc(wp, m.a * m.Sj1 * m.SE1));
    const Z dA = zsub(zadd(zmul(dwb, D2), zsc(zmul(wb, D), 2.0)), zc(m.a * m.Sj1 * m.SE1, 0.0));
    // S and S'
    const Z wb2K = zsub(zmul(wb, wb), zc(K2, 0.0));
    const double sb = m.b * m.Sj2;
    const Z S = zsub(zmul(wb2K, D), zsc(zsub(zsc(wb, m.SE2), zsc(cs, m.SB3s * m.kE1 * m.v0)), sb));
    const Z dS = zsub(zadd(zsc(zmul(zmul(wb, dwb), D), 2.0), wb2K),
                      zsc(zsub(zsc(dwb, m.SE2), zsc(dcs, m.SB3s * m.kE1 * m.v0)), sb));
    // C and C'
    const double c1 = m.b * m.Sj1 * m.SE1 * kE2s * (m.v0 * m.v0 - 1.0);
    const double c2 = m.b * m.Sj2 * m.SE2 * kE2s;
    const double c3 = m.b * m.Sj1 * m.kE2 * m.k2 * m.SE2 * m.kE1 * m.v0;
    const double c4 = m.b * m.Sj1 * m.kE2 * m.k2 * m.SB3s * m.v0 * m.v0;
    const Z C = zsub(zadd(zadd(zsc(wp, c1), zsc(D, c2)), zc(c3, 0.0)), zsc(zmul(cs, wb), c4));
    const Z dC = zsub(zc(c1 + c2, 0.0), zsc(zadd(zmul(dcs, wb), zmul(cs, dwb)), c4));
    *g = zadd(zmul(A, S), zmul(C, D));
    if (dg) *dg = zadd(zadd(zadd(zmul(dA, S), zmul(A, dS)), zmul(dC, D)), C);
}

// Winding number of G along a closed polyline given by point(i), i = 0..n (point(n) =
// point(0)), with the number of points raised until no phase step exceeds 0.5 rad.
// Returns -1 if no sampling up to kMaxWind points resolves it (a zero on the path).
constexpr int kMaxWind = 1 << 13;
template <typename Path>
__device__ int winding(const NciMode& m, Path path, int n0) {
    for (int n = n0; n <= kMaxWind; n *= 4) {
        Z g0;
        nci_G(m, path(0, n), &g0, nullptr);
        const Z gs = g0;
        double tot = 0.0;
        bool ok = true;
        for (int i = 1; i <= n && ok; i++) {
            Z g1;
            if (i == n) g1 = gs;
            else nci_G(m, path(i, n), &g1, nullptr);
            // arg(g1 / g0) = atan2(Im(g1 conj g0), Re(g1 conj g0))
            const double re = g1.re * g0.re + g1.im * g0.im, im = g1.im * g0.re - g1.re * g0.im;
            if (re == 0.0 && im == 0.0) { ok = false; break; }
            const double d = atan2(im, re);
            if (fabs(d) > 0.5) ok = false;
            tot += d;
            g0 = g1;
        }
        if (ok) return (int)llround(tot / (2.0 * 3.14159265358979323846));
    }
    return -1;
}

__device__ int winding_circle(const NciMode& m, Z c, double r) {
    return winding(m, [&](int i, int n) {
        double s, co;
        sincospi(2.0 * (double)i / (double)n, &s, &co);
        return zc(c.re + r * co, c.im + r * s);
    }, 64);
}
__device__ int winding_rect(const NciMode& m, double x0, double x1, double y0, double y1) {
    return winding(m, [&](int i, int n) {
        // n points, n/4 per edge, counter-clockwise from (x0, y0)
        const int q = n / 4, e = i / q;
        const double t = (double)(i - e * q) / (double)q;
        if (e == 0) return zc(x0 + (x1 - x0) * t, y0);
        if (e == 1) return zc(x1, y0 + (y1 - y0) * t);
        if (e == 2) return zc(x1 - (x1 - x0) * t, y1);
        if (e == 3) return zc(x0, y1 - (y1 - y0) * t);
        return zc(x0, y0);
    }, 128);
}

// Newton's method on G deflated by the nf zeros in r[]; true if it converges to w.
__device__ bool newton_deflated(const NciMode& m, Z w, const Z* r, int nf, Z* out) {
    for (int it = 0; it < 80; it++) {
        Z g, dg;
        nci_G(m, w, &g, &dg);
        if (g.re == 0.0 && g.im == 0.0) { *out = w; return true; }
        Z q = zdiv(dg, g);                               // G'/G
        for (int j = 0; j < nf; j++) q = zsub(q, zdiv(zc(1.0, 0.0), zsub(w, r[j])));
        if (q.re == 0.0 && q.im == 0.0) return false;
        const Z step = zdiv(zc(1.0, 0.0), q);
        w = zsub(w, step);
        if (!(isfinite(w.re) && isfinite(w.im))) return false;
        if (zabs(step) <= 1e-14 * fmax(1.0, zabs(w))) { *out = w; return true; }
    }
    return false;
}

// Plain Newton's method for one zero inside a rectangle.
__device__ bool newton_in(const NciMode& m, Z w, double x0, double x1, double y0, double y1, Z* out) {
    Z r;
    if (!newton_deflated(m, w, nullptr, 0, &r)) return false;
    if (r.re < x0 || r.re > x1 || r.im < y0 || r.im > y1) return false;
    *out = r;
    return true;
}

constexpr int kMaxRoots = 16;   // zeros kept per (sample, alias); more is reported as an error
constexpr int kStack = 96;      // subdivision stack entries

// the cubic a x^3 + b x^2 + c x + d = 0 (a != 0) by the trigonometric / Cardano forms
__device__ void cubic_roots(double a, double b, double c, double d, Z r[3]) {
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
}

// one row of the samples array
struct NciSample { double dt, dx1, dx2, gamma, wp2, filt_kc, filt_w, k1, k2, kmod_l, kmod_u, kmod_max; };

__device__ double filt_factor(const NciSample& s) {
    if (!(s.filt_kc > 0.0 && s.filt_kc < 1.0)) return 1.0;
    const double pi = 3.14159265358979323846, kn = pi / s.dx1, k = fabs(s.k1);
    const double kc = s.filt_kc * kn, w = s.filt_w * kn;
    if (k <= kc - 0.5 * w) return 1.0;
    if (k >= kc + 0.5 * w) return 0.0;
    const double c = cos(0.5 * pi * (k - kc + 0.5 * w) / w);
    return c * c;
}

// [k]E1 = [k]B1: k1 plus the Sec. 4 raised-cosine bump between kmod_l and kmod_u (fractions of 2 pi/dx1)
__device__ double k_eff(const NciSample& s) {
    double k = s.k1;
    if (s.kmod_max != 0.0) {
        const double pi = 3.14159265358979323846, kg = 2.0 * pi / s.dx1;
        const double kl = s.kmod_l * kg, ku = s.kmod_u * kg, km = 0.5 * (kl + ku), a = fabs(s.k1);
        if (a >= kl && a <= ku) {
            const double c = cos(0.5 * pi * (a - km) / (kl - km));
            k += copysign(s.kmod_max * kg * c * c, s.k1);
        }
    }
    return k;
}

// error bits of k_nci (the kernel's *err)
enum : int { NCI_ETOOMANY = 1, NCI_EUNRESOLVED = 2 };

__global__ void k_nci(const NciSample* __restrict__ smp, int64_t n, int order, int correct_j1,
                      const int* __restrict__ alias, int n_alias, double* __restrict__ growth, double2* __restrict__ root,
                      int max_out, double2* __restrict__ roots_out, int* __restrict__ count_out, int* __restrict__ err) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= n * n_alias) return;
    const int64_t i = tid / n_alias;
    const int ai = (int)(tid % n_alias);
    const NciSample s = smp[i];
    const double pi = 3.14159265358979323846;
    NciMode m;
    m.h = 0.5 * s.dt;
    m.v0 = sqrt(1.0 - 1.0 / (s.gamma * s.gamma));
    m.mu = alias[2 * ai];
    const int nu1 = alias[2 * ai + 1];
    m.wg = 2.0 * pi / s.dt;
    const double sgnmu = (m.mu & 1) ? -1.0 : 1.0;
    m.a = s.wp2 / (s.gamma * s.gamma * s.gamma) * sgnmu;
    m.b = s.wp2 / s.gamma * sgnmu;
    m.k2 = s.k2;
    m.k1a = s.k1 + nu1 * 2.0 * pi / s.dx1;
    const double s1 = dsinc(0.5 * m.k1a * s.dx1), s2 = dsinc(0.5 * s.k2 * s.dx2);
    double sl1 = s1, sl2 = s2, sm1 = 1.0, sm2 = 1.0;                 // orders l + 1 and l
    for (int q = 0; q < order; q++) { sl1 *= s1; sl2 *= s2; sm1 *= s1; sm2 *= s2; }
    const double sgn = (nu1 & 1) ? -1.0 : 1.0;
    m.kE1 = k_eff(s);
    m.kE2 = sin(0.5 * s.k2 * s.dx2) / (0.5 * s.dx2);
    m.SE1 = sl1 * sl2 * sgn;
    m.SE2 = sl1 * sl2;
    m.SB3s = sl1 * sl2 * sgn;
    const double F = filt_factor(s);
    const double corr = (correct_j1 && s.k1 != 0.0) ? dsinc(0.5 * s.k1 * s.dx1) * s.k1 / m.kE1 : 1.0;
    m.Sj1 = sm1 * sl2 * sgn * F * corr;
    m.Sj2 = sl1 * sm2 * F;

    const Z c = zc(m.k1a * m.v0 - m.mu * m.wg, 0.0);                // the resonance
    const double rho = cbrt(s.wp2 / s.gamma);
    Z r[kMaxRoots];
    int nf = 0, N = 0, e = 0;
    if (rho > 0.0) {
        N = winding_circle(m, c, rho);
        if (N < 0 || N > kMaxRoots) { e |= (N < 0) ? NCI_EUNRESOLVED : NCI_ETOOMANY; N = 0; }
    }
    // ---- seeds: the cubic's roots (Eq. asym1, v0 -> 1 in k~1), the resonance, rings in the disk
    if (N > 0) {
        const double kt = m.k1a - m.mu * m.wg, hh = m.h;
        const double xi0 = sin(kt * hh) / hh, xi1 = cos(kt * hh), ze0 = cos(kt * hh), ze1 = -sin(kt * hh) * hh;
        const double kE1 = m.kE1, kE2 = m.kE2, SB = m.SB3s;
        const double A2 = 2.0 * xi0 * xi0 * xi0 * xi1;
        const double B2 = xi0 * xi0 * (xi0 * xi0 - kE1 * kE1 - kE2 * kE2 - m.b * m.Sj2 * (m.SE2 * xi1 - ze1 * SB * kE1));
        const double C2 = m.b * (xi0 * xi0 * m.Sj2 * (ze0 * SB * kE1 - m.SE2 * xi0) - xi1 * m.Sj1 * kE2 * m.k2 * m.SE2 * kE1
                                 + xi0 * kE2 * (m.Sj2 * m.SE2 * kE2 - m.Sj1 * m.k2 * ze1 * SB * xi0));
        const double D2 = m.b * xi0 * kE2 * m.k2 * m.Sj1 * (m.SE2 * kE1 - ze0 * SB * xi0);
        constexpr int kRing = 8;
        const int nseed = 4 + 3 * kRing;
        Z cub[3];
        const bool have_cubic = A2 != 0.0;
        if (have_cubic) cubic_roots(A2, B2, C2, D2, cub);
        for (int q = 0; q < nseed && nf < N; q++) {
            Z w0;
            if (q < 3) {
                if (!have_cubic) continue;
                w0 = zc(c.re + cub[q].re, cub[q].im);
                if (zabs(zsub(w0, c)) >= rho) continue;
            } else if (q == 3) {
                w0 = zc(c.re + 1e-6 * rho, 1e-7 * rho);
            } else {
                const int ring = (q - 4) / kRing, k = (q - 4) % kRing;
                const double rr = rho * (0.15 + 0.3 * ring);
                double sn, cs;
                sincospi((2.0 * k + 0.5 * ring) / kRing, &sn, &cs);
                w0 = zc(c.re + rr * cs, c.im + rr * sn);
            }
            Z w;
            if (!newton_deflated(m, w0, r, nf, &w)) continue;
            if (zabs(zsub(w, c)) >= rho) continue;
            r[nf++] = w;
        }
    }
    // ---- the rest by argument-principle subdivision of a rectangle enclosing the disk
    if (nf < N) {
        nf = 0;
        const double fr[4][2] = {{0.4871, 0.5317}, {0.4413, 0.5689}, {0.5593, 0.4231}, {0.3917, 0.6143}};
        const double hmin = fmax(1e-12 * rho, 1e-9 * fmax(1.0, zabs(c)));
        double x0 = c.re - rho, x1 = c.re + 1.0007 * rho, y0 = c.im - 1.0003 * rho, y1 = c.im + 1.0011 * rho;
        const int Nr = winding_rect(m, x0, x1, y0, y1);
        if (Nr < 0) e |= NCI_EUNRESOLVED;
        struct Rect { double x0, x1, y0, y1; int N; };
        Rect st[kStack];
        int sp = 0;
        if (Nr > 0) st[sp++] = Rect{x0, x1, y0, y1, Nr};
        while (sp > 0) {
            const Rect q = st[--sp];
            if (q.N == 1) {
                Z w;
                if (newton_in(m, zc(q.x0 + fr[0][0] * (q.x1 - q.x0), q.y0 + fr[0][1] * (q.y1 - q.y0)), q.x0, q.x1, q.y0, q.y1, &w)) {
                    if (zabs(zsub(w, c)) < rho) {
                        if (nf < kMaxRoots) r[nf++] = w;
                        else e |= NCI_ETOOMANY;
                    }
                    continue;
                }
            }
            if (fmax(q.x1 - q.x0, q.y1 - q.y0) < hmin) {          // a cluster below resolution
                const Z w = zc(0.5 * (q.x0 + q.x1), 0.5 * (q.y0 + q.y1));
                if (zabs(zsub(w, c)) < rho)
                    for (int k = 0; k < q.N; k++) {
                        if (nf < kMaxRoots) r[nf++] = w;
                        else e |= NCI_ETOOMANY;
                    }
                continue;
            }
            bool split = false;
            for (int f = 0; f < 4 && !split; f++) {
                const double xm = q.x0 + fr[f][0] * (q.x1 - q.x0), ym = q.y0 + fr[f][1] * (q.y1 - q.y0);
                const Rect kid[4] = {{q.x0, xm, q.y0, ym, 0}, {xm, q.x1, q.y0, ym, 0}, {q.x0, xm, ym, q.y1, 0}, {xm, q.x1, ym, q.y1, 0}};
                int ns[4], tot = 0;
                bool ok = true;
                for (int k = 0; k < 4 && ok; k++) {
                    ns[k] = winding_rect(m, kid[k].x0, kid[k].x1, kid[k].y0, kid[k].y1);
                    ok = ns[k] >= 0;
                    tot += ns[k];
                }
                if (!ok || tot != q.N) continue;
                split = true;
                for (int k = 0; k < 4; k++) {
                    if (ns[k] == 0) continue;
                    if (sp >= kStack) { e |= NCI_EUNRESOLVED; break; }
                    st[sp] = kid[k];
                    st[sp].N = ns[k];
                    sp++;
                }
            }
            if (!split) e |= NCI_EUNRESOLVED;
        }
    }
    double best = 0.0;
    Z broot = c;
    for (int k = 0; k < nf; k++)
        if (r[k].im > best) { best = r[k].im; broot = r[k]; }
    growth[tid] = best;
    if (root) root[tid] = make_double2(broot.re, broot.im);
    if (count_out) count_out[tid] = nf;
    if (roots_out)
        for (int k = 0; k < max_out; k++) roots_out[tid * max_out + k] = k < nf ? make_double2(r[k].re, r[k].im) : make_double2(0.0, 0.0);
    if (e && err) atomicOr(err, e);
}

static hyb_status nci_launch(const double* samples, int64_t n, int order, int correct_j1, const int* alias, int n_alias,
                             double* growth, double* root, int max_out, double* roots_out, int* count_out, int* err,
                             void* stream) {
    if (!samples || !alias || !growth || n < 0 || n_alias < 1 || order < 1 || order > 3 || max_out < 0) {
        set_error("hyb_nci_growth: bad arguments");
        return HYB_EINVAL;
    }
    if (n == 0) return HYB_OK;
    const int64_t total = n * n_alias;
    const int thr = 64;
    k_nci<<<(unsigned)((total + thr - 1) / thr), thr, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const NciSample*>(samples), n, order, correct_j1, alias, n_alias, growth,
        reinterpret_cast<double2*>(root), max_out, reinterpret_cast<double2*>(roots_out), count_out, err);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" hyb_status hyb_nci_growth(const double* samples, int64_t n, int order, int correct_j1,
                                     const int* alias, int n_alias, double* growth, double* root, void* stream) {
    return nci_launch(samples, n, order, correct_j1, alias, n_alias, growth, root, 0, nullptr, nullptr, nullptr, stream);
}

extern "C" hyb_status hyb_nci_roots(const double* samples, int64_t n, int order, int correct_j1, const int* alias,
                                    int n_alias, int max_roots, double* roots, int* count, double* growth, int* err,
                                    void* stream) {
    if (!roots || !count || max_roots < 1) {
        set_error("hyb_nci_roots: bad arguments");
        return HYB_EINVAL;
    }
    return nci_launch(samples, n, order, correct_j1, alias, n_alias, growth, nullptr, max_roots, roots, count, err, stream);
}
