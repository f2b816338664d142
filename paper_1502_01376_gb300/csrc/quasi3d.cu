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

#include <type_traits>
#include <vector>

#include <algorithm>

#include "hyb_internal.cuh"
#include "packed_dev.cuh"

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
    float2* tw2k = nullptr;   // stage twiddles of k_cfft2048 (FP32, nz = 2048 only)
    cplx<T>* spec = nullptr;  // [12][nr][nz]: E, B, J spectra, then the advanced B (E^{n+1} replaces J)
};

struct QPtrs { void* p[9]; };
// the arrays of up to kQModes modes advanced by one launch (modes of equal nz = 2048, nr, dr):
// mode q's field f at p[9 q + f], its spectra at spec[q]
constexpr int kQModes = 8;
struct QMulti { void* p[kQModes * 9]; float2* spec[kQModes]; int nm; };

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

// ---------------------------------------------------------------- nz = 2048, FP32: register-resident rows
// X[k] = sum_j x[j] W^{jk}, W = exp(-2 pi i / 2048), factored 8 x 8 x 8 x 4 with k = k1 + 8 k2 + 64 k3 + 512 k4:
//   S1  thread t:            DFT8 over n of x[t + 256 n] -> k1, times W_2048^{t k1}      -> A(k1, t)
//   S2  (t0, k1) = (t & 31, t >> 5):  DFT8 over t1 of A(k1, t0 + 32 t1) -> k2, times W_256^{t0 k2}
//   S3  (u0, k1, k2) = (t & 3, (t >> 2) & 7, t >> 5):  DFT8 over u1 of A'(k1, k2, u0 + 4 u1) -> k3,
//       times W_32^{u0 k3}
//   S4  the 512 (k1, k2, k3) in two halves:  DFT4 over u0 -> k4, written to X[k1 + 8 k2 + 64 k3 + 512 k4]
// Exchange layouts (float2 units): A(k1, t) at 256 k1 + t; A'(k1, k2, t0) at 260 k1 + 32 k2 + t0;
// A''(k1, k2, k3, u0) at 516 u0 + 64 k3 + k1 + 8 k2 (in the A buffer).  With 8-byte accesses a half-warp
// of every exchange reaches 16 different bank pairs; global loads and stores are row-contiguous per warp.
// The inverse uses the conjugate twiddles and scales by 1/2048.  One row per 256-thread block
// iteration; persistent, the next row's points held in registers while the current one is transformed.
constexpr int kQ2k = 2048;
constexpr int kQ2kA = 2064, kQ2kB = 2080;
constexpr int kQ2kTw = 7 * 256 + 7 * 32 + 7 * 4;     // stage twiddles, in the order the threads read them

template <bool INV>
__device__ __forceinline__ float2 q2k_tw(float2 a, float2 w) {
    return INV ? make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y))
               : make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

template <bool INV>
__global__ void __launch_bounds__(256, 2) k_cfft2048(const __grid_constant__ QMulti io, int nr, int nf,
                                                     const float2* __restrict__ tw) {
    __shared__ __align__(16) float2 bufA[kQ2kA];
    __shared__ __align__(16) float2 bufB[kQ2kB];
    const int t = threadIdx.x;
    const int64_t per = (int64_t)nr * nf, total = per * io.nm;
    float2 w1[8], w2[8], w3[8], nx[8];
#pragma unroll
    for (int k = 1; k < 8; k++) {
        w1[k] = tw[(k - 1) * 256 + t];
        w2[k] = tw[1792 + (k - 1) * 32 + (t & 31)];
        w3[k] = tw[2016 + (k - 1) * 4 + (t & 3)];
    }
    // row j of the launch: mode q, field f, radial row r; its spectrum row is jj of mode q
    auto src_of = [&](int64_t j) -> const float2* {
        const int q = (int)(j / per);
        const int64_t jj = j - q * per;
        const int f = (int)(jj / nr);
        const int64_t r = jj - (int64_t)f * nr;
        return INV ? io.spec[q] + jj * kQ2k : reinterpret_cast<const float2*>(io.p[9 * q + f]) + r * kQ2k;
    };
    auto fetch = [&](int64_t j) {
        const float2* x = src_of(j);
#pragma unroll
        for (int n = 0; n < 8; n++) nx[n] = __ldcs(x + t + 256 * n);
    };
    int64_t j = blockIdx.x;
    if (j < total) fetch(j);
    for (; j < total; j += gridDim.x) {
        float2 v[8];
#pragma unroll
        for (int n = 0; n < 8; n++) v[n] = nx[n];
        if (j + gridDim.x < total) fetch(j + gridDim.x);
        // S1
        dft8x<INV>(v);
#pragma unroll
        for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], w1[k]);
        __syncthreads();                 // the previous row's S4 has read the A buffer
#pragma unroll
        for (int k = 0; k < 8; k++) bufA[256 * k + t] = v[k];
        __syncthreads();
        // S2
        {
            const int t0 = t & 31, k1 = t >> 5;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = bufA[256 * k1 + t0 + 32 * n];
            dft8x<INV>(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], w2[k]);
#pragma unroll
            for (int k = 0; k < 8; k++) bufB[260 * k1 + 32 * k + t0] = v[k];
        }
        __syncthreads();
        // S3
        {
            const int u0 = t & 3, k1 = (t >> 2) & 7, k2 = t >> 5;
#pragma unroll
            for (int n = 0; n < 8; n++) v[n] = bufB[260 * k1 + 32 * k2 + u0 + 4 * n];
            dft8x<INV>(v);
#pragma unroll
            for (int k = 1; k < 8; k++) v[k] = q2k_tw<INV>(v[k], w3[k]);
#pragma unroll
            for (int k = 0; k < 8; k++) bufA[516 * u0 + 64 * k + k1 + 8 * k2] = v[k];
        }
        __syncthreads();
        // S4
        float2* X;
        {
            const int q = (int)(j / per);
            const int64_t jj = j - q * per;
            const int f = (int)(jj / nr);
            const int64_t r = jj - (int64_t)f * nr;
            X = INV ? reinterpret_cast<float2*>(io.p[9 * q + f]) + r * kQ2k : io.spec[q] + jj * kQ2k;
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int it = t + 256 * h;      // k1 + 8 k2 + 64 k3
            float2 a0 = bufA[it], a1 = bufA[516 + it], a2 = bufA[1032 + it], a3 = bufA[1548 + it];
            dft4x<INV>(a0, a1, a2, a3);
            if (INV) {
                const float s = 1.0f / (float)kQ2k;
                a0 = vmul(a0, make_float2(s, s)); a1 = vmul(a1, make_float2(s, s));
                a2 = vmul(a2, make_float2(s, s)); a3 = vmul(a3, make_float2(s, s));
            }
            __stcs(X + it, a0);
            __stcs(X + it + 512, a1);
            __stcs(X + it + 1024, a2);
            __stcs(X + it + 1536, a3);
        }
    }
}

// stage twiddles of k_cfft2048, W_N^e = exp(-2 pi i e / N), in the order above
static std::vector<float2> cfft2048_twiddles() {
    std::vector<float2> w(kQ2kTw);
    const double pi = 3.14159265358979323846;
    auto W = [&](int e, int N) { const double a = 2.0 * pi * e / N; return make_float2((float)cos(a), (float)-sin(a)); };
    for (int k = 1; k < 8; k++) {
        for (int t = 0; t < 256; t++) w[(k - 1) * 256 + t] = W(t * k, 2048);
        for (int t = 0; t < 32; t++) w[1792 + (k - 1) * 32 + t] = W(t * k, 256);
        for (int t = 0; t < 4; t++) w[2016 + (k - 1) * 4 + t] = W(t * k, 32);
    }
    return w;
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
struct QLeap { cplx<T>* spec[kQModes]; const QTab<T>* tab[kQModes]; T dt[kQModes]; int m[kQModes]; };

template <typename T>
__global__ void __launch_bounds__(kQThreads) k_qleap(const __grid_constant__ QLeap<T> ql, int nz, int nr, T dr) {
    using C = cplx<T>;
    cplx<T>* __restrict__ spec = ql.spec[blockIdx.z];               // mode of this block
    const QTab<T>* __restrict__ tab = ql.tab[blockIdx.z];
    const T dt = ql.dt[blockIdx.z];
    const int m = ql.m[blockIdx.z];
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
    if (std::is_same<T, float>::value && nz == kQ2k) {
        const std::vector<float2> w2k = cfft2048_twiddles();
        HYB_CUDA_TRY(cudaMalloc(&P->tw2k, sizeof(float2) * w2k.size()));
        HYB_CUDA_TRY(cudaMemcpy(P->tw2k, w2k.data(), sizeof(float2) * w2k.size(), cudaMemcpyHostToDevice));
    }
    const size_t smem = sizeof(C) * 2 * fpad_size((size_t)fft_rows_per_block(nz) * nz);
    HYB_CUDA_TRY(cudaFuncSetAttribute(k_qfft<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HYB_CUDA_TRY(cudaFuncSetAttribute(k_qfft<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return HYB_OK;
}

// one step of the modes gs[0 .. n - 1] (n = 1, or modes that qualify for quasi3d_advance_many)
// on stream st: z transform of E, B, j, the leapfrog, inverse of the advanced E, B
template <typename T>
static hyb_status step_modes(hyb_grid* const* gs, int n, cudaStream_t st) {
    using C = cplx<T>;
    hyb_grid* g = gs[0];
    QPlan<T>* P = reinterpret_cast<QPlan<T>*>(g->qtab);
    const hyb_grid_desc& d = g->d;
    const int nz = d.n1, nr = d.n2;
    QLeap<T> ql{};
    for (int q = 0; q < n; q++) {
        QPlan<T>* Pq = reinterpret_cast<QPlan<T>*>(gs[q]->qtab);
        ql.spec[q] = Pq->spec;
        ql.tab[q] = Pq->tab;
        ql.dt[q] = (T)gs[q]->d.dt;
        ql.m[q] = gs[q]->d.azimuthal_m;
    }
    if (P->tw2k) {
        QMulti fin{}, fout{};
        for (int q = 0; q < n; q++) {
            for (int c = 0; c < 3; c++) {
                fin.p[9 * q + c] = gs[q]->E[c]; fin.p[9 * q + 3 + c] = gs[q]->B[c]; fin.p[9 * q + 6 + c] = gs[q]->J[c];
                fout.p[9 * q + c] = gs[q]->E[c]; fout.p[9 * q + 3 + c] = gs[q]->B[c];
            }
            QPlan<T>* Pq = reinterpret_cast<QPlan<T>*>(gs[q]->qtab);
            fin.spec[q] = reinterpret_cast<float2*>(Pq->spec);
            fout.spec[q] = reinterpret_cast<float2*>(Pq->spec + 6 * (int64_t)nr * nz);
        }
        fin.nm = fout.nm = n;
        const int res = resident_grid((const void*)k_cfft2048<false>, 256, 0);
        k_cfft2048<false><<<(unsigned)std::min<int64_t>(res, (int64_t)n * 9 * nr), 256, 0, st>>>(fin, nr, 9, P->tw2k);
        const dim3 mgrid((unsigned)((nz + kQThreads - 1) / kQThreads), (unsigned)nr, (unsigned)n);
        k_qleap<T><<<mgrid, kQThreads, 0, st>>>(ql, nz, nr, (T)d.dx2);
        const int res2 = resident_grid((const void*)k_cfft2048<true>, 256, 0);
        k_cfft2048<true><<<(unsigned)std::min<int64_t>(res2, (int64_t)n * 6 * nr), 256, 0, st>>>(fout, nr, 6, P->tw2k);
    } else {
        const int RB = fft_rows_per_launch(nz, (int64_t)nr * 6), nblk = (nr + RB - 1) / RB;
        const size_t smem = sizeof(C) * 2 * fpad_size((size_t)RB * nz);
        QPtrs fin{}, fout{};
        for (int c = 0; c < 3; c++) { fin.p[c] = g->E[c]; fin.p[3 + c] = g->B[c]; fin.p[6 + c] = g->J[c]; }
        for (int c = 0; c < 3; c++) { fout.p[c] = g->E[c]; fout.p[3 + c] = g->B[c]; }
        const int gf = std::min(9 * nblk, resident_grid((const void*)k_qfft<T, false>, kQThreads, smem));
        const int gi = std::min(6 * nblk, resident_grid((const void*)k_qfft<T, true>, kQThreads, smem));
        k_qfft<T, false><<<gf, kQThreads, smem, st>>>(fin, P->spec, nz, nr, 9, P->tw, RB);
        const dim3 mgrid((unsigned)((nz + kQThreads - 1) / kQThreads), (unsigned)nr, 1u);
        k_qleap<T><<<mgrid, kQThreads, 0, st>>>(ql, nz, nr, (T)d.dx2);
        k_qfft<T, true><<<gi, kQThreads, smem, st>>>(fout, P->spec + 6 * (int64_t)nr * nz, nz, nr, 6, P->tw, RB);
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

template <typename T>
static hyb_status advance_t(hyb_grid* g, int nsteps) {
    for (int s = 0; s < nsteps; s++) {
        if (g->ev_start) HYB_CUDA_TRY(cudaEventRecord(g->ev_start, g->stream));
        hyb_status st = step_modes<T>(&g, 1, g->stream);
        if (st != HYB_OK) return st;
        if (g->ev_stop) HYB_CUDA_TRY(cudaEventRecord(g->ev_stop, g->stream));
    }
    return HYB_OK;
}

bool quasi3d_can_batch(const hyb_grid* a, const hyb_grid* b) {
    return a->d.dims == 20 && b->d.dims == 20 && a->d.precision == 32 && b->d.precision == 32 && a->d.n1 == 2048 &&
           b->d.n1 == 2048 && a->d.n2 == b->d.n2 && a->d.dx2 == b->d.dx2;
}

hyb_status quasi3d_advance_many(hyb_grid* const* gs, int n, cudaStream_t st) {
    for (int i = 0; i < n; i += kQModes) {
        const int m = std::min(kQModes, n - i);
        hyb_status r = step_modes<float>(gs + i, m, st);
        if (r != HYB_OK) return r;
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
        cudaFree(P->tab); cudaFree(P->tw); cudaFree(P->tw2k); cudaFree(P->spec); delete P;
    } else {
        QPlan<double>* P = reinterpret_cast<QPlan<double>*>(g->qtab);
        cudaFree(P->tab); cudaFree(P->tw); cudaFree(P->tw2k); cudaFree(P->spec); delete P;
    }
    g->qtab = nullptr;
}

hyb_status quasi3d_advance(hyb_grid* g, int nsteps) {
    return g->d.precision == 32 ? advance_t<float>(g, nsteps) : advance_t<double>(g, nsteps);
}

}  // namespace hyb
