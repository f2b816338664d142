// hyb_internal.cuh -- grid object and helpers shared by the libhyb.so
// translation units (not part of the public ABI; see include/hyb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

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

// ---------------------------------------------------------------- shared-memory radix-2 Stockham FFT
template <typename C>
__device__ __forceinline__ void stockham_radix2(C*& src, C*& dst, int M, const C* __restrict__ twM, bool inverse) {
    // natural-order in, natural-order out; one __syncthreads per stage
    for (int Ns = 1; Ns < M; Ns <<= 1) {
        const int tstride = M / (2 * Ns);
        for (int j = threadIdx.x; j < (M >> 1); j += blockDim.x) {
            const int k = j & (Ns - 1);
            C a = src[j], b = src[j + (M >> 1)];
            C w = twM[k * tstride];
            b = inverse ? cmulc(b, w) : cmul(b, w);
            const int o = ((j - k) << 1) + k;
            dst[o] = cadd(a, b);
            dst[o + Ns] = csub(a, b);
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }
}


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
    double* diag_work = nullptr;   // diagnostics: 2 spectral FP64 arrays + 1 real FP64 array
    size_t diag_bytes = 0;
    double* diag_acc = nullptr;    // 16 FP64 accumulators
    int* dflag = nullptr;          // device data-error flag
    hyb::FusedPlan* fused = nullptr;
    void* qtab = nullptr;          // quasi-3D per-mode tables (device)
    void* dft = nullptr;           // path 3: DFT-GEMM matrices and buffers
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // optional kernel timing events
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
hyb_status generic_launches_per_step();

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

// quasi-3D azimuthal-mode path (quasi3d.cu)
hyb_status quasi3d_create(hyb_grid* g);
void quasi3d_destroy(hyb_grid* g);
hyb_status quasi3d_advance(hyb_grid* g, int nsteps);

// x1 transform as a split-BF16 DFT-GEMM on the tensor cores (dftgemm.cu)
hyb_status dftgemm_create(hyb_grid* g);
void dftgemm_destroy(hyb_grid* g);
hyb_status dftgemm_forward(hyb_grid* g, const float* const* fields, int nf, float2* spec);
hyb_status dftgemm_inverse(hyb_grid* g, const float2* spec, int nf, float* const* fields);

// deposit (deposit.cu)
template <typename T>
hyb_status deposit(hyb_grid* g, const int32_t* cell, const T* off_old, const T* off_new, const T* v3,
                   const T* q, int64_t np, int order);

// diagnostics (diag.cu)
template <typename T> hyb_status diag(hyb_grid* g, double out[9]);

}  // namespace hyb
