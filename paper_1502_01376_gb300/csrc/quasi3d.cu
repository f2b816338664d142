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

#include "q3d_body.cuh"

namespace hyb {


template <typename T>
struct QPlan {
    QTab<T>* tab = nullptr;
    cplx<T>* tw = nullptr;    // stockham_twiddles(nz)
    float2* tw2k = nullptr;   // stage twiddles of k_cfft2048 (FP32, nz = 2048 only)
    cplx<T>* spec = nullptr;  // [12][nr][nz]: E, B, J spectra, then the advanced B (E^{n+1} replaces J)
};

struct QPtrs { void* p[9]; };

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

template <bool INV>
__global__ void __launch_bounds__(256, 2) k_cfft2048(const __grid_constant__ QMulti io, int nr, int nf,
                                                     const float2* __restrict__ tw) {
    __shared__ __align__(16) float2 bufA[kQ2kA];
    __shared__ __align__(16) float2 bufB[kQ2kB];
    cfft2048_body<INV, false>(io, nr, nf, tw, blockIdx.x, gridDim.x, threadIdx.x, bufA, bufB, 0);
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

// one leapfrog step per (axial mode, radial row, mode): grid (nz / kQThreads, nr, modes)
template <typename T>
__global__ void __launch_bounds__(kQThreads) k_qleap(const __grid_constant__ QLeap<T> ql, int nz, int nr, T dr) {
    qleap_body<T>(ql, nz, nr, dr, (int)(blockIdx.x * blockDim.x + threadIdx.x), (int)blockIdx.y, (int)blockIdx.z);
}

// the same for FP32 modes with nz = 2048 in columns (qleap_column: a block takes 256 axial modes of a
// chunk of `rows` radial rows of one mode, the rows staged by bulk copy); persistent over the
// ncol x nch columns
constexpr int kQColSmem = 2 * 9 * 256 * 8 + 2 * 8 + 4;
__global__ void __launch_bounds__(256) k_qleap_col(const __grid_constant__ QLeap<float> ql, int nr, float dr, int nm,
                                                   int nch, int rows, int* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    float2* st = reinterpret_cast<float2*>(sm);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * 9 * 256 * 8);
    volatile int* abort = reinterpret_cast<volatile int*>(sm + 2 * 9 * 256 * 8 + 16);
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(bars), 1);
        mbar_init(smem_addr(bars + 1), 1);
        *abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    constexpr int nkb = kQ2k / 256;
    const int ncol = nkb * nm;
    uint32_t ph = 0;
    for (int u = blockIdx.x; u < ncol * nch; u += gridDim.x) {
        const int col = u % ncol, ch = u / ncol;
        const int j0 = ch * rows, j1 = min(nr, j0 + rows);
        if (j0 < j1)
            qleap_column<float>(ql, kQ2k, nr, dr, col % nkb, col / nkb, j0, j1, threadIdx.x, st, smem_addr(bars),
                                smem_addr(bars + 1), ph, 1, err, abort);
    }
    if (*abort && threadIdx.x == 0) {
        if (ph & 4u) mbar_drain(smem_addr(bars), (ph & 1u) ^ 1u);
        if (ph & 8u) mbar_drain(smem_addr(bars + 1), ((ph >> 1) & 1u) ^ 1u);
    }
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

// the arguments of the FP32 nz = 2048 stages for the modes gs[0 .. n - 1] (n <= kQModes, pairwise
// quasi3d_can_batch): the forward transform reads E, B, j of every mode into its spectra, the
// inverse writes the advanced E, B spectra (slots 6 .. 11) back to E, B
hyb_status quasi3d_step_args(hyb_grid* const* gs, int n, Q3Args* out) {
    if (n < 1 || n > kQModes || gs[0]->d.precision != 32) { set_error("quasi3d_step_args: bad modes"); return HYB_EINVAL; }
    const QPlan<float>* P = reinterpret_cast<const QPlan<float>*>(gs[0]->qtab);
    if (!P || !P->tw2k) { set_error("quasi3d_step_args: not the nz = 2048 FP32 path"); return HYB_EINVAL; }
    const int nz = gs[0]->d.n1, nr = gs[0]->d.n2;
    Q3Args a{};
    for (int q = 0; q < n; q++) {
        for (int c = 0; c < 3; c++) {
            a.fin.p[9 * q + c] = gs[q]->E[c]; a.fin.p[9 * q + 3 + c] = gs[q]->B[c]; a.fin.p[9 * q + 6 + c] = gs[q]->J[c];
            a.fout.p[9 * q + c] = gs[q]->E[c]; a.fout.p[9 * q + 3 + c] = gs[q]->B[c];
        }
        QPlan<float>* Pq = reinterpret_cast<QPlan<float>*>(gs[q]->qtab);
        a.fin.spec[q] = reinterpret_cast<float2*>(Pq->spec);
        a.fout.spec[q] = reinterpret_cast<float2*>(Pq->spec + 6 * (int64_t)nr * nz);
        a.ql.spec[q] = Pq->spec;
        a.ql.tab[q] = Pq->tab;
        a.ql.dt[q] = (float)gs[q]->d.dt;
        a.ql.m[q] = gs[q]->d.azimuthal_m;
    }
    a.fin.nm = a.fout.nm = n;
    a.tw2k = P->tw2k;
    a.nr = nr;
    a.nm = n;
    a.dr = (float)gs[0]->d.dx2;
    *out = a;
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
        Q3Args a{};
        hyb_status hs = quasi3d_step_args(gs, n, &a);
        if (hs != HYB_OK) return hs;
        const int res = resident_grid((const void*)k_cfft2048<false>, 256, 0);
        k_cfft2048<false><<<(unsigned)std::min<int64_t>(res, (int64_t)n * 9 * nr), 256, 0, st>>>(a.fin, nr, 9, a.tw2k);
        // the leapfrog in columns, about as many as the resident blocks
        HYB_CUDA_TRY(func_attr_once((const void*)k_qleap_col, cudaFuncAttributeMaxDynamicSharedMemorySize, kQColSmem));
        const int resl = resident_grid((const void*)k_qleap_col, 256, kQColSmem);
        const int ncol = (kQ2k / 256) * n, nch = std::max(1, std::min(nr, resl / ncol)), rows = (nr + nch - 1) / nch;
        k_qleap_col<<<(unsigned)std::min(resl, ncol * nch), 256, kQColSmem, st>>>(a.ql, nr, a.dr, n, nch, rows, g->dflag);
        const int res2 = resident_grid((const void*)k_cfft2048<true>, 256, 0);
        k_cfft2048<true><<<(unsigned)std::min<int64_t>(res2, (int64_t)n * 6 * nr), 256, 0, st>>>(a.fout, nr, 6, a.tw2k);
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
