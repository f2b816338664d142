// hyb_internal.cuh -- grid object and helpers shared by the libhyb.so
// translation units (not part of the public ABI; see include/hyb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/hyb.h"

namespace hyb {

// ---------------------------------------------------------------- complex ops
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mkc(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) { return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) { return mkc<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mkc<C>(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mkc<C>(a.x * s, a.y * s); }

// ---------------------------------------------------------------- shared-memory Stockham FFT (radix 8, 4, 2)
// Small DFTs in natural order; INV uses W = exp(+2 pi i / R) (no scaling).
template <typename C, bool INV>
__device__ __forceinline__ C rot_i(C a) { return INV ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x); }   // times -i (fwd) / +i (inv)

template <typename C, bool INV>
__device__ __forceinline__ void sdft2(C* x) { const C t = x[0]; x[0] = cadd(t, x[1]); x[1] = csub(t, x[1]); }

template <typename C, bool INV>
__device__ __forceinline__ void sdft4(C& x0, C& x1, C& x2, C& x3) {
    const C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = rot_i<C, INV>(csub(x1, x3));
    x0 = cadd(a, c); x2 = csub(a, c); x1 = cadd(b, d); x3 = csub(b, d);
}

template <typename C, bool INV>
__device__ __forceinline__ void sdft8(C* x) {
    using T = decltype(C::x);
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    sdft4<C, INV>(e0, e1, e2, e3);
    sdft4<C, INV>(o0, o1, o2, o3);
    const T h = (T)0.70710678118654752440;
    // o1 W8^1, o2 W8^2, o3 W8^3 (conjugate roots for the inverse)
    o1 = INV ? mkc<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mkc<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    o2 = rot_i<C, INV>(o2);
    o3 = INV ? mkc<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mkc<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

// Shared-memory position of element i of the FFT buffers: one padding element after every
// sixteen, so that the stride-8 scatter of a radix-8 pass spreads over all banks while
// contiguous accesses stay (nearly) conflict-free.
__host__ __device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
// elements of a padded buffer holding n values
__host__ __device__ __forceinline__ size_t fpad_size(size_t n) { return n + n / 16 + 1; }

// One radix-R Stockham pass over nrow rows of M points (rows contiguous): butterfly j of a
// row (0 <= j < M/R, k = j mod Ns) takes src[j + r M/R] W_{R Ns}^{r k}, r = 0..R-1, does an
// R-point DFT over r and writes output r to dst[(j - k) R + k + r Ns].  The twiddles come from
// the pass-ordered table of stockham_twiddles, W_{R Ns}^{r k} at Ns - 1 + (r - 1) Ns + k, so that
// the lanes of a warp (consecutive k) read consecutive entries.
template <typename C, int R, bool INV>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst, int lgM, int lgNs, int nrow,
                                              const C* __restrict__ tw) {
    constexpr int lgR = (R == 8) ? 3 : (R == 4) ? 2 : 1;
    const int M = 1 << lgM, Ns = 1 << lgNs;
    const int lgnb = lgM - lgR, nb = 1 << lgnb;
    // padded positions: when the element stride is a multiple of 16, fpad(a + r s) = fpad(a) + r (s + s / 16)
    const bool rstride = (nb & 15) == 0, wstride = (Ns & 15) == 0;
    const int nbp = nb + (nb >> 4), nsp = Ns + (Ns >> 4);
    for (int q = threadIdx.x; q < (nrow << lgnb); q += blockDim.x) {
        const int row = q >> lgnb, j = q & (nb - 1), k = j & (Ns - 1);
        const int base = row * M;
        const int ra = fpad(base + j);
        C x[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            x[r] = src[rstride ? ra + r * nbp : fpad(base + j + r * nb)];
            if (r > 0 && Ns > 1) {
                const C w = tw[Ns - 1 + (r - 1) * Ns + k];
                x[r] = INV ? cmulc(x[r], w) : cmul(x[r], w);
            }
        }
        if (R == 8) sdft8<C, INV>(x);
        else if (R == 4) sdft4<C, INV>(x[0], x[1], x[2], x[3]);
        else sdft2<C, INV>(x);
        const int o = base + (j - k) * R + k;
        const int wa = fpad(o);
#pragma unroll
        for (int r = 0; r < R; r++) dst[wstride ? wa + r * nsp : fpad(o + r * Ns)] = x[r];
    }
}

// natural-order in, natural-order out FFT of nrow rows of M = 2^m points held in shared
// memory (src, padded positions fpad(row * M + j)); radix-8 passes then one radix-4 or
// radix-2 pass; one __syncthreads per pass.  On return src points at the result.
// tw: stockham_twiddles(M).
template <typename C, bool INV>
__device__ __forceinline__ void stockham_rows(C*& src, C*& dst, int M, int nrow, const C* __restrict__ tw) {
    const int lgM = 31 - __clz(M);
    int lgNs = 0;
    while (lgNs + 3 <= lgM) {
        stockham_pass<C, 8, INV>(src, dst, lgM, lgNs, nrow, tw);
        __syncthreads();
        C* t = src; src = dst; dst = t;
        lgNs += 3;
    }
    if (lgNs + 2 <= lgM) {
        stockham_pass<C, 4, INV>(src, dst, lgM, lgNs, nrow, tw);
        __syncthreads();
        C* t = src; src = dst; dst = t;
    } else if (lgNs + 1 <= lgM) {
        stockham_pass<C, 2, INV>(src, dst, lgM, lgNs, nrow, tw);
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }
}

constexpr int kTw8 = 504;   // entries of ModeTables::tw8

// x1 wavenumbers of mode kappa in FP64: k1 = 2 pi kappa / (n1 dx1); the Yee symbol
// [k]1 = sin(k1 dx1/2)/(dx1/2); and the wavenumber the advance differentiates with
// (Sec. 2.1: [k]1 replaced by k1; the Yee symbol itself in Yee-recovery mode; k1 plus the
// raised-cosine bump of Sec. 4 between kmod_l and kmod_u, fractions of k_g1 = 2 pi/dx1).
// One definition for the host tables and for tables built on the device.
struct ModeK { double k1, kfd, keff; };
__host__ __device__ inline ModeK mode_k(int kappa, int n1, double dx1, int yee_mode, double kmod_l, double kmod_u,
                                        double kmod_max) {
    const double pi = 3.14159265358979323846, kg = 2.0 * pi / dx1;
    ModeK m;
    m.k1 = kg * (double)kappa / (double)n1;
    m.kfd = sin(0.5 * m.k1 * dx1) / (0.5 * dx1);
    m.keff = m.k1;
    if (yee_mode) {
        m.keff = m.kfd;
    } else if (kmod_max != 0.0) {
        const double kl = kmod_l * kg, ku = kmod_u * kg, km = 0.5 * (kl + ku);
        if (m.k1 >= kl && m.k1 <= ku) {
            const double c = cos(0.5 * pi * (m.k1 - km) / (kl - km));
            m.keff += kmod_max * kg * c * c;
        }
    }
    return m;
}
// Eq. currentcorrection factor of mode kappa ([k]1 of the finite difference over the
// advance's wavenumber; 1 at kappa = 0)
__host__ __device__ inline double mode_corr(int kappa, const ModeK& m) { return kappa == 0 ? 1.0 : m.kfd / m.keff; }

// Entry i of stockham_twiddles(M) as W = exp(-2 pi i num/den): the pass with span Ns and
// radix R holds W_{R Ns}^{r k} at Ns - 1 + (r - 1) Ns + k.  Returns num = 0, den = 1 for
// the one entry no pass uses.
__host__ __device__ inline void stockham_tw_frac(int M, int i, int* num, int* den) {
    int lgM = 0;
    while ((1 << lgM) < M) lgM++;
    int lgNs = 0;
    *num = 0;
    *den = 1;
    while (lgNs < lgM) {
        const int lgR = (lgNs + 3 <= lgM) ? 3 : (lgNs + 2 <= lgM) ? 2 : 1;
        const int Ns = 1 << lgNs, R = 1 << lgR;
        if (i >= Ns - 1 && i < R * Ns - 1) {
            const int q = i - (Ns - 1), r = 1 + q / Ns, k = q % Ns;
            *num = r * k;
            *den = R * Ns;
            return;
        }
        lgNs += lgR;
    }
}
// Entry i of ModeTables::tw8 as W = exp(-2 pi i num/den)
__host__ __device__ inline void tw8_frac(int i, int* num, int* den) {
    if (i < 448) { *num = (i % 64) * (1 + i / 64); *den = 512; }
    else { *num = ((i - 448) % 8) * (1 + (i - 448) / 8); *den = 64; }
}

// The twiddles of the passes stockham_rows makes for M points, in pass order: the pass with span
// Ns and radix R holds W_{R Ns}^{r k} (r = 1..R-1, k < Ns) at Ns - 1 + (r - 1) Ns + k, so the
// passes fill entries 0..M-2 (computed in FP64, rounded once).
template <typename C>
inline std::vector<C> stockham_twiddles(int M) {
    std::vector<C> tw((size_t)M);
    for (int i = 0; i < M; i++) {
        int num, den;
        stockham_tw_frac(M, i, &num, &den);
        const double a = -2.0 * 3.14159265358979323846 * (double)num / (double)den;
        tw[(size_t)i] = mkc<C>((decltype(C::x))std::cos(a), (decltype(C::x))std::sin(a));
    }
    return tw;
}

// ModeTables::tw8 for M = 512 (computed in FP64, rounded once)
template <typename C>
inline std::vector<C> tw8_table() {
    std::vector<C> tw(kTw8);
    for (int i = 0; i < kTw8; i++) {
        int num, den;
        tw8_frac(i, &num, &den);
        const double a = -2.0 * 3.14159265358979323846 * (double)num / (double)den;
        tw[(size_t)i] = mkc<C>((decltype(C::x))std::cos(a), (decltype(C::x))std::sin(a));
    }
    return tw;
}

// rows of M points one block of 256 threads transforms together (one radix-8 pass then
// has about 256 butterflies) ...
__host__ __device__ __forceinline__ int fft_rows_per_block(int M) { return M >= 2048 ? 1 : 2048 / M; }
// ... reduced for small launches so that there are at least about 600 blocks (4 per SM)
__host__ __forceinline__ int fft_rows_per_launch(int M, int64_t total_rows) {
    int rb = fft_rows_per_block(M);
    while (rb > 1 && total_rows / rb < 600) rb >>= 1;
    return rb;
}

// Persistent launches of the shared-memory complex row FFTs (quasi-3D): a block takes the
// row blocks i = blockIdx.x, blockIdx.x + gridDim.x, ... and, when a row block is at most
// kPrefetchPts points per thread, holds the next block's points in registers while it
// transforms the current one.
constexpr int kPrefetchPts = 8;
// blocks of `threads` threads with `smem` bytes of dynamic shared memory that fit on the
// current device at once (cached per device, kernel and size)
int resident_grid(const void* kernel, int threads, size_t smem);
// cudaFuncSetAttribute(kernel, attr, value) on the current device, once per device (a
// function attribute set on one device does not carry over to another)
cudaError_t func_attr_once(const void* kernel, cudaFuncAttribute attr, int value);

// ---------------------------------------------------------------- tables
// Per-mode tables for kappa = 0..n1/2, computed in FP64 on the host and rounded once.
template <typename T>
struct ModeTables {
    cplx<T>* S = nullptr;     // c dt sigma+ = c dt i [k]1 exp(+i k1 dx1/2)
    T* cj1 = nullptr;         // ampere dt F (corr if correct_j1): coefficient of j1 in Ampere
    T* cj = nullptr;          // ampere dt F: coefficient of j2, j3
    T* corr = nullptr;        // Eq. currentcorrection factor alone
    T* filt = nullptr;        // Sec. 4 form factor alone
    cplx<T>* twM = nullptr;   // W_M^j = exp(-2 pi i j / M), j < M, M = n1/2
    cplx<T>* twN = nullptr;   // W_N^k = exp(-2 pi i k / n1), k < M
    cplx<T>* sgp = nullptr;   // sigma+ (without c dt), for diagnostics
    cplx<T>* twS = nullptr;   // stockham_twiddles(M): the shared-memory row FFTs
    // M = 512 only (n1 = 1024, factored 8 x 8 x 8): the twiddles of the first two stages in the
    // order the threads read them, [(k - 1) 64 + t] = W_512^{t k} (k = 1..7, t < 64), then
    // [448 + (k - 1) 8 + t0] = W_64^{t0 k} (t0 < 8)
    cplx<T>* tw8 = nullptr;
};

struct FusedPlan;   // defined in fused_api.cuh

}  // namespace hyb

struct hyb_grid {
    hyb_grid_desc d;
    cudaStream_t stream = nullptr;
    int device = 0;
    int path = 1;
    int64_t rows = 0;        // n2 * n3
    int64_t cells = 0;
    int nk = 0;              // n1/2 + 1
    // bound caller arrays
    void* E[3] = {nullptr, nullptr, nullptr};
    void* B[3] = {nullptr, nullptr, nullptr};
    void* J[3] = {nullptr, nullptr, nullptr};
    void* rho = nullptr;
    bool bound = false;
    // tables in run precision and in FP64 (diagnostics)
    hyb::ModeTables<float> tf;
    hyb::ModeTables<double> td;
    // scratch (library-owned)
    void* spec = nullptr;          // three-pass path: 9 spectral arrays [9][rows][nk] complex of run precision
    size_t spec_bytes = 0;
    int spec_fields = 0;           // 9 (three-pass or k1-resident) or 3 (fused path: j only)
    // k1-resident state (hyb_set_resident): the spectra of E, B in spec carry over between steps;
    // res_stale: the next step first imports them from the bound real arrays
    bool resident = false;
    bool res_stale = true;
    double* diag_work = nullptr;   // diagnostics: 2 spectral FP64 arrays + 1 real FP64 array
    size_t diag_bytes = 0;
    double* diag_acc = nullptr;    // 16 FP64 accumulators
    int* dflag = nullptr;          // device data-error flag
    hyb::FusedPlan* fused = nullptr;
    void* qtab = nullptr;          // quasi-3D per-mode tables (device)
    void* dft = nullptr;           // path 3: DFT-GEMM matrices and buffers
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // optional kernel timing events
    // one three-pass (or quasi-3D) step captured as a CUDA graph and replayed per step, so
    // that small grids do not pay a launch per kernel; re-captured after hyb_bind_fields
    cudaGraphExec_t step_exec = nullptr;
    bool step_dirty = true;
};

namespace hyb {

void set_error(const char* fmt, ...);
hyb_status cuda_fail(cudaError_t e, const char* what);

#define HYB_CUDA_TRY(call)                                         \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return ::hyb::cuda_fail(e__, #call); \
    } while (0)

// three-pass path (generic.cu)
template <typename T> hyb_status generic_advance(hyb_grid* g, int nsteps);
template <typename T> hyb_status generic_process_current(hyb_grid* g, bool corr, bool filt);
// k1-resident state (three-pass path): import E, B into the spectra; B^n = B^{n-1/2} + Faraday/2
// from the spectra into the real arrays Bh (the PIC step's gather)
template <typename T> hyb_status generic_resident_import(hyb_grid* g);
template <typename T> hyb_status generic_b_half(hyb_grid* g, void* const Bh[3]);
int generic_launches_per_step(const hyb_grid* g);

// batched real FFT along x1 (generic.cu); in: rows of n1 reals of Tin;
// out: rows of n1/2+1 complex of T (strides in elements)
template <typename Tin, typename T>
cudaError_t rfft_rows(const Tin* in, cplx<T>* out, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s);
template <typename T, typename Tout>
cudaError_t irfft_rows(const cplx<T>* in, Tout* out, int n1, int64_t rows, const ModeTables<T>& t, cudaStream_t s);

// fused FP32 2D path (fused2d.cu)
bool fused_supported(const hyb_grid_desc& d);
hyb_status fused_create(hyb_grid* g);
void fused_destroy(hyb_grid* g);
hyb_status fused_advance(hyb_grid* g, int nsteps);
int fused_launches_per_step(const hyb_grid* g);
bool fused_epoch_launches(const hyb_grid* g);
const char* fused_step_kernel(const hyb_grid* g);   // name of the kernel one step launches

// quasi-3D azimuthal-mode path (quasi3d.cu)
hyb_status quasi3d_create(hyb_grid* g);
void quasi3d_destroy(hyb_grid* g);
hyb_status quasi3d_advance(hyb_grid* g, int nsteps);
// one step of several FP32 modes with nz = 2048 and equal nr, dr (quasi3d_can_batch pairwise
// with the first) in three launches on stream st
bool quasi3d_can_batch(const hyb_grid* a, const hyb_grid* b);
hyb_status quasi3d_advance_many(hyb_grid* const* gs, int n, cudaStream_t st);

// x1 transform as a split-BF16 DFT-GEMM on the tensor cores (dftgemm.cu)
hyb_status dftgemm_create(hyb_grid* g);
void dftgemm_destroy(hyb_grid* g);
hyb_status dftgemm_forward(hyb_grid* g, const float* const* fields, int nf, float2* spec);
hyb_status dftgemm_inverse(hyb_grid* g, const float2* spec, int nf, float* const* fields);

// deposit (deposit.cu)
template <typename T>
hyb_status deposit(hyb_grid* g, const int32_t* cell, const T* off_old, const T* off_new, const T* v3,
                   const T* q, int64_t np, int order);

// field gather and Boris push (push.cu)
template <typename T>
hyb_status push(hyb_grid* g, int32_t* cell, T* off, T* u, const T* qm, T* off_new, T* v3, int64_t np, int order);
// the same with the fields given explicitly (E[3], B[3] of the grid's shape and precision)
template <typename T>
hyb_status push_fields(hyb_grid* g, void* const E[3], void* const B[3], int32_t* cell, T* off, T* u, const T* qm,
                       T* off_new, T* v3, int64_t np, int order);

// diagnostics (diag.cu)
template <typename T> hyb_status diag(hyb_grid* g, double out[9]);

}  // namespace hyb
