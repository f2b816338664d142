// quasi3d.cu -- hybrid solver for one azimuthal mode m of the quasi-3D
// geometry (Sec. 5): complex fields F_m(r, z) (the amplitude of exp(i m phi)),
// z (x1) spectral with the 2D solver's sigma+/- symbols and the j_z
// correction, r (x2) by the Yee differences of the cylindrical curl
//   (curl A)_r = (i m / r) A_z - dA_phi/dz,  (curl A)_phi = dA_r/dz - dA_z/dr,
//   (curl A)_z = (1/r) d(r A_phi)/dr - (i m / r) A_r,
// on the 2D staggering with x1 = z, x2 = r (E_z, E_r, E_phi, B_z, B_r, B_phi
// in the E1..B3 slots), r_j = j dr.  Axis: E_z(0) from the circulation of
// B_phi round a disc of radius dr/2 for m = 0, else 0; E_phi(0), B_r(0) only
// for m = 1 (with dB_z/dr(0) = 2 B_z(dr/2)/dr and (i m/r) E_z -> i m E_z(dr)/dr),
// else 0.  A perfect conductor at r = n_r dr.  Three launches per step: complex
// FFT along z of the nine arrays, the leapfrog (Faraday then Ampere) per (r, k_z)
// in one kernel, inverse FFT of the six advanced spectra.
#include <math.h>

#include <vector>

#include <algorithm>

#include "hyb_internal.cuh"

namespace hyb {

template <typename T>
struct QTab {
    cplx<T> sp;   // sigma+ = i k e^{+i k dz/2}
    cplx<T> sm;   // sigma- = i k e^{-i k dz/2}
    T cjz;        // ampere dt F corr
    T cj;         // ampere dt F
};

template <typename T>
struct QPlan {
    QTab<T>* tab = nullptr;
    cplx<T>* tw = nullptr;    // stockham_twiddles(nz)
    cplx<T>* spec = nullptr;  // [12][nr][nz]: E, B, J spectra, then the advanced B (E^{n+1} replaces J)
};

struct QPtrs { void* p[9]; };

constexpr int kQThreads = 256;

// i m / r times a
template <typename C>
__device__ __forceinline__ C imr(C a, decltype(C::x) m_over_r) { return mkc<C>(-m_over_r * a.y, m_over_r * a.x); }

// complex transforms along z of row blocks of RB rows (block i: field i / nblk); persistent, the
// next block's points held in registers while the current one is transformed (RB nz <= 2048)
template <typename T, bool INV>
__global__ void __launch_bounds__(kQThreads) k_qfft(QPtrs io, cplx<T>* __restrict__ spec, int nz, int nr, int nf,
                                                   const cplx<T>* __restrict__ tw, int RB) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* const src0 = reinterpret_cast<C*>(smem_raw);
    C* const dst0 = src0 + fpad_size((size_t)RB * nz);
    const int nblk = (nr + RB - 1) / RB, total = nblk * nf;
    const bool pf = RB * nz <= kPrefetchPts * kQThreads;
    // forward: fields -> spectral scratch; inverse: scratch -> fields (scaled by 1/nz)
    auto in_of = [&](int f, int row0) -> const C* {
        return INV ? spec + ((int64_t)f * nr + row0) * nz : reinterpret_cast<const C*>(io.p[f]) + (int64_t)row0 * nz;
    };
    C nx[kPrefetchPts];
    auto fetch = [&](int i) {
        const int f = i / nblk, row0 = (i - f * nblk) * RB;
        const int cnt = ((nr - row0) < RB ? (nr - row0) : RB) * nz;
        const C* x = in_of(f, row0);
#pragma unroll
        for (int u = 0; u < kPrefetchPts; u++) {
            const int q = threadIdx.x + u * kQThreads;
            if (q < cnt) nx[u] = x[q];
        }
    };
    int i = blockIdx.x;
    if (pf && i < total) fetch(i);
    for (; i < total; i += gridDim.x) {
        const int f = i / nblk, row0 = (i - f * nblk) * RB;
        const int nrow = (nr - row0) < RB ? (nr - row0) : RB;
        __syncthreads();                                   // the previous block has read its result
        if (pf) {
#pragma unroll
            for (int u = 0; u < kPrefetchPts; u++) {
                const int q = threadIdx.x + u * kQThreads;
                if (q < nrow * nz) src0[fpad(q)] = nx[u];
            }
            if (i + gridDim.x < total) fetch(i + gridDim.x);
        } else {
            const C* x = in_of(f, row0);
            for (int q = threadIdx.x; q < nrow * nz; q += blockDim.x) src0[fpad(q)] = x[q];
        }
        __syncthreads();
        C* src = src0;
        C* dst = dst0;
        stockham_rows<C, INV>(src, dst, nz, nrow, tw);
        if (INV) {
            C* x = reinterpret_cast<C*>(io.p[f]) + (int64_t)row0 * nz;
            const T inv = (T)1 / (T)nz;
            for (int q = threadIdx.x; q < nrow * nz; q += blockDim.x) x[q] = cscale(src[fpad(q)], inv);
        } else {
            C* X = spec + ((int64_t)f * nr + row0) * nz;
            for (int q = threadIdx.x; q < nrow * nz; q += blockDim.x) X[q] = src[fpad(q)];
        }
    }
}

template <typename T>
struct QB { cplx<T> z, r, p; };

// Faraday for axial mode k at radial row j: B^{n+1/2} from B^{n-1/2} at j and E^n at rows j and j+1
// (tangential E vanishes on the conducting wall r = nr dr; on the axis B_r follows the m rules)
template <typename T>
__device__ __forceinline__ QB<T> qfaraday_at(const cplx<T>* __restrict__ spec, int64_t fs, int nz, int nr, int j, int k,
                                             cplx<T> sp, T dt, T dr, int m) {
    using C = cplx<T>;
    const C* Ez = spec; const C* Er = spec + fs; const C* Ep = spec + 2 * fs;
    const C* Bz = spec + 3 * fs; const C* Br = spec + 4 * fs; const C* Bp = spec + 5 * fs;
    const T ri = (T)j * dr, rh = ((T)j + (T)0.5) * dr, rup = (T)(j + 1) * dr;
    const T mT = (T)m;
    const int64_t i = (int64_t)j * nz + k, iu = i + nz;
    const C ez = Ez[i], er = Er[i], ep = Ep[i];
    const C ezu = (j + 1 < nr) ? Ez[iu] : mkc<C>((T)0, (T)0);
    const C epu = (j + 1 < nr) ? Ep[iu] : mkc<C>((T)0, (T)0);
    C cr;
    if (j > 0) cr = csub(imr(ez, mT / ri), cmul(sp, ep));
    else if (m == 1) cr = csub(imr(Ez[nz + k], mT / dr), cmul(sp, ep));
    else cr = mkc<C>((T)0, (T)0);
    const C cp = csub(cmul(sp, er), cscale(csub(ezu, ez), (T)1 / dr));
    const C cz = csub(cscale(csub(cscale(epu, rup), cscale(ep, ri)), (T)1 / (rh * dr)), imr(er, mT / rh));
    QB<T> b;
    b.z = csub(Bz[i], cscale(cz, dt));
    b.r = (j == 0 && m != 1) ? mkc<C>((T)0, (T)0) : csub(Br[i], cscale(cr, dt));
    b.p = csub(Bp[i], cscale(cp, dt));
    return b;
}

// one leapfrog step per (axial mode k, radial row j) on the spectra [E, B, J] (slots 0..8): Faraday at
// rows j and j-1 (the latter recomputed, so no launch boundary is needed between the halves), then
// Ampere at row j.  E^{n+1} goes to the J slots 6..8 (J at row j is read by this thread only) and
// B^{n+1/2} to slots 9..11; slots 0..5 are only read, so neighbouring threads see the old values.
template <typename T>
__global__ void __launch_bounds__(kQThreads) k_qleap(cplx<T>* __restrict__ spec, int nz, int nr, const QTab<T>* __restrict__ tab,
                                                    T dt, T dr, int m) {
    using C = cplx<T>;
    const int j = blockIdx.y;                                        // radial row
    const int k = blockIdx.x * blockDim.x + threadIdx.x;             // axial mode
    if (k >= nz) return;
    const int64_t fs = (int64_t)nr * nz, i = (int64_t)j * nz + k;
    const C* Ez = spec; const C* Er = spec + fs; const C* Ep = spec + 2 * fs;
    C* Jz = spec + 6 * fs; C* Jr = spec + 7 * fs; C* Jp = spec + 8 * fs;
    C* Bn = spec + 9 * fs;
    const T ri = (T)j * dr, rh = ((T)j + (T)0.5) * dr, rd = ((T)j - (T)0.5) * dr;
    const T mT = (T)m;
    const QTab<T> q = tab[k];
    const QB<T> b = qfaraday_at<T>(spec, fs, nz, nr, j, k, q.sp, dt, dr, m);
    const C cr = csub(imr(b.z, mT / rh), cmul(q.sm, b.p));
    C cp, cz;
    if (j > 0) {
        const QB<T> bd = qfaraday_at<T>(spec, fs, nz, nr, j - 1, k, q.sp, dt, dr, m);
        cp = csub(cmul(q.sm, b.r), cscale(csub(b.z, bd.z), (T)1 / dr));
        cz = csub(cscale(csub(cscale(b.p, rh), cscale(bd.p, rd)), (T)1 / (ri * dr)), imr(b.r, mT / ri));
    } else {
        cp = (m == 1) ? csub(cmul(q.sm, b.r), cscale(b.z, (T)2 / dr)) : mkc<C>((T)0, (T)0);
        cz = (m == 0) ? cscale(b.p, (T)4 / dr) : mkc<C>((T)0, (T)0);
    }
    C er = csub(cadd(Er[i], cscale(cr, dt)), cscale(Jr[i], q.cj));
    C ep = csub(cadd(Ep[i], cscale(cp, dt)), cscale(Jp[i], q.cj));
    C ez = csub(cadd(Ez[i], cscale(cz, dt)), cscale(Jz[i], q.cjz));
    if (j == 0 && m != 0) ez = mkc<C>((T)0, (T)0);
    if (j == 0 && m != 1) ep = mkc<C>((T)0, (T)0);
    Jz[i] = ez;
    Jr[i] = er;
    Jp[i] = ep;
    Bn[i] = b.z;
    Bn[fs + i] = b.r;
    Bn[2 * fs + i] = b.p;
}

template <typename T>
static hyb_status create_t(hyb_grid* g) {
    using C = cplx<T>;
    const hyb_grid_desc& d = g->d;
    const int nz = d.n1, nr = d.n2;
    QPlan<T>* P = new QPlan<T>();
    g->qtab = P;
    const double pi = 3.14159265358979323846;
    std::vector<QTab<T>> tab(nz);
    const bool filt_on = d.filt_kc > 0.0 && d.filt_kc < 1.0;
    for (int k = 0; k < nz; k++) {
        const int kap = (k <= nz / 2) ? k : k - nz;                  // Nyquist taken as +nz/2
        const double kk = 2.0 * pi * kap / (nz * d.dx1);
        const double ph = 0.5 * kk * d.dx1;
        tab[k].sp = mkc<C>((T)(-kk * sin(ph)), (T)(kk * cos(ph)));
        tab[k].sm = mkc<C>((T)(kk * sin(ph)), (T)(kk * cos(ph)));
        const double corr = (kap == 0 || !d.correct_j1) ? 1.0 : sin(ph) / ph;
        double F = 1.0;
        if (filt_on) {
            const double kn = pi / d.dx1, a = fabs(kk), kc = d.filt_kc * kn, w = d.filt_w * kn;
            if (w <= 0.0) F = a <= kc ? 1.0 : 0.0;
            else if (a <= kc - 0.5 * w) F = 1.0;
            else if (a >= kc + 0.5 * w) F = 0.0;
            else { const double c = cos(0.5 * pi * (a - kc + 0.5 * w) / w); F = c * c; }
        }
        tab[k].cjz = (T)(d.ampere * d.dt * F * corr);
        tab[k].cj = (T)(d.ampere * d.dt * F);
    }
    const std::vector<C> tw = stockham_twiddles<C>(nz);
    HYB_CUDA_TRY(cudaMalloc(&P->tab, sizeof(QTab<T>) * nz));
    HYB_CUDA_TRY(cudaMemcpy(P->tab, tab.data(), sizeof(QTab<T>) * nz, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMalloc(&P->tw, sizeof(C) * nz));
    HYB_CUDA_TRY(cudaMemcpy(P->tw, tw.data(), sizeof(C) * nz, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMalloc(&P->spec, sizeof(C) * 12 * (size_t)nr * nz));
    const size_t smem = sizeof(C) * 2 * fpad_size((size_t)fft_rows_per_block(nz) * nz);
    HYB_CUDA_TRY(cudaFuncSetAttribute(k_qfft<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HYB_CUDA_TRY(cudaFuncSetAttribute(k_qfft<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return HYB_OK;
}

template <typename T>
static hyb_status advance_t(hyb_grid* g, int nsteps) {
    using C = cplx<T>;
    QPlan<T>* P = reinterpret_cast<QPlan<T>*>(g->qtab);
    const hyb_grid_desc& d = g->d;
    const int nz = d.n1, nr = d.n2;
    const int RB = fft_rows_per_launch(nz, (int64_t)nr * 6), nblk = (nr + RB - 1) / RB;
    const size_t smem = sizeof(C) * 2 * fpad_size((size_t)RB * nz);
    QPtrs fin{}, fout{};
    for (int c = 0; c < 3; c++) { fin.p[c] = g->E[c]; fin.p[3 + c] = g->B[c]; fin.p[6 + c] = g->J[c]; }
    for (int c = 0; c < 3; c++) { fout.p[c] = g->E[c]; fout.p[3 + c] = g->B[c]; }
    const int gf = std::min(9 * nblk, resident_grid((const void*)k_qfft<T, false>, kQThreads, smem));
    const int gi = std::min(6 * nblk, resident_grid((const void*)k_qfft<T, true>, kQThreads, smem));
    for (int s = 0; s < nsteps; s++) {
        if (g->ev_start) HYB_CUDA_TRY(cudaEventRecord(g->ev_start, g->stream));
        k_qfft<T, false><<<gf, kQThreads, smem, g->stream>>>(fin, P->spec, nz, nr, 9, P->tw, RB);
        const dim3 mgrid((unsigned)((nz + kQThreads - 1) / kQThreads), (unsigned)nr);   // one thread per (mode, row)
        k_qleap<T><<<mgrid, kQThreads, 0, g->stream>>>(P->spec, nz, nr, P->tab, (T)d.dt, (T)d.dx2, d.azimuthal_m);
        k_qfft<T, true><<<gi, kQThreads, smem, g->stream>>>(fout, P->spec + 6 * (int64_t)nr * nz, nz, nr, 6, P->tw, RB);
        HYB_CUDA_TRY(cudaGetLastError());
        if (g->ev_stop) HYB_CUDA_TRY(cudaEventRecord(g->ev_stop, g->stream));
    }
    return HYB_OK;
}

hyb_status quasi3d_create(hyb_grid* g) {
    return g->d.precision == 32 ? create_t<float>(g) : create_t<double>(g);
}

void quasi3d_destroy(hyb_grid* g) {
    if (!g->qtab) return;
    if (g->d.precision == 32) {
        QPlan<float>* P = reinterpret_cast<QPlan<float>*>(g->qtab);
        cudaFree(P->tab); cudaFree(P->tw); cudaFree(P->spec); delete P;
    } else {
        QPlan<double>* P = reinterpret_cast<QPlan<double>*>(g->qtab);
        cudaFree(P->tab); cudaFree(P->tw); cudaFree(P->spec); delete P;
    }
    g->qtab = nullptr;
}

hyb_status quasi3d_advance(hyb_grid* g, int nsteps) {
    return g->d.precision == 32 ? advance_t<float>(g, nsteps) : advance_t<double>(g, nsteps);
}

}  // namespace hyb
