// diag.cu -- FP64 diagnostics of the bound fields: field energies, the
// discrete div B of the hybrid scheme and the Gauss's-law residual of Sec. 2.3,
//   G = sigma- E1 + d2- E2 [+ d3- E3] - ampere F rho,
// whose time derivative vanishes when the corrected (and filtered) current
// drives Ampere's law.  The x1 derivatives go through FP64 row FFTs.
#include "hyb_internal.cuh"

namespace hyb {

constexpr int kDiagThreads = 256;

// |x| of a finite double, as an ordered integer key for atomicMax
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(fabs(x));
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kDiagThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (kDiagThreads / 32) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

struct Ptr6 { const void* p[6]; };

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_energy(Ptr6 f, int64_t n, double* __restrict__ acc) {
    const T* x = reinterpret_cast<const T*>(f.p[blockIdx.y]);
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(acc + blockIdx.y, s);
}

// spec *= sym (sign = +1: sigma+, -1: sigma- = -conj(sigma+))
__global__ void k_mul_sigma(double2* __restrict__ spec, int nk, int64_t rows, const double2* __restrict__ sgp, int sign) {
    const int64_t r = blockIdx.x;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        double2 s = sgp[k];
        if (sign < 0) s = make_double2(-s.x, s.y);
        spec[r * nk + k] = cmul(spec[r * nk + k], s);
    }
}

// a -= coef * F * b
__global__ void k_sub_filtered(double2* __restrict__ a, const double2* __restrict__ b, int nk, int64_t rows,
                               const double* __restrict__ filt, double coef) {
    const int64_t r = blockIdx.x;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const double f = coef * filt[k];
        double2 v = a[r * nk + k], w = b[r * nk + k];
        a[r * nk + k] = make_double2(v.x - f * w.x, v.y - f * w.y);
    }
}

// D += dir * (d2 f2 [+ d3 f3]), dir = +1: forward differences (div B), -1: backward (Gauss)
template <typename T>
__global__ void __launch_bounds__(kDiagThreads) k_add_fd(double* __restrict__ D, const T* __restrict__ f2, const T* __restrict__ f3,
                                                         int n1, int n2, int n3, double inv2, double inv3, int forward,
                                                         double* __restrict__ acc, unsigned long long* __restrict__ amax) {
    const int64_t n = (int64_t)n1 * n2 * n3;
    double ss = 0.0;
    unsigned long long m = 0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int i1 = (int)(i % n1);
        const int64_t rr = i / n1;
        const int i2 = (int)(rr % n2), i3 = (int)(rr / n2);
        double v = D[i];
        if (forward) {
            const int j2 = i2 + 1 == n2 ? 0 : i2 + 1;
            v += ((double)f2[((int64_t)i3 * n2 + j2) * n1 + i1] - (double)f2[i]) * inv2;
            if (f3) {
                const int j3 = i3 + 1 == n3 ? 0 : i3 + 1;
                v += ((double)f3[((int64_t)j3 * n2 + i2) * n1 + i1] - (double)f3[i]) * inv3;
            }
        } else {
            const int j2 = i2 == 0 ? n2 - 1 : i2 - 1;
            v += ((double)f2[i] - (double)f2[((int64_t)i3 * n2 + j2) * n1 + i1]) * inv2;
            if (f3) {
                const int j3 = i3 == 0 ? n3 - 1 : i3 - 1;
                v += ((double)f3[i] - (double)f3[((int64_t)j3 * n2 + i2) * n1 + i1]) * inv3;
            }
        }
        D[i] = v;
        ss += v * v;
        unsigned long long kk = abs_key(v);
        m = kk > m ? kk : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(amax, m);
    ss = block_sum(ss);
    if (threadIdx.x == 0) atomicAdd(acc, ss);
}

template <typename T>
hyb_status diag(hyb_grid* g, double out[9]) {
    const hyb_grid_desc& d = g->d;
    const int64_t rows = g->rows, cells = g->cells;
    const int nk = g->nk, n1 = d.n1, n3 = d.dims == 3 ? d.n3 : 1;
    const size_t spec_bytes = (size_t)rows * nk * sizeof(double2);
    if (!g->diag_work) {
        g->diag_bytes = 2 * spec_bytes + (size_t)cells * sizeof(double);
        cudaError_t e = cudaMalloc(&g->diag_work, g->diag_bytes);
        if (e != cudaSuccess) { g->diag_work = nullptr; return cuda_fail(e, "cudaMalloc(diagnostics scratch)"); }
    }
    double2* s1 = reinterpret_cast<double2*>(g->diag_work);
    double2* s2 = reinterpret_cast<double2*>(reinterpret_cast<char*>(g->diag_work) + spec_bytes);
    double* D = reinterpret_cast<double*>(reinterpret_cast<char*>(g->diag_work) + 2 * spec_bytes);
    double* acc = g->diag_acc;                                         // [0..5] energies, [6] gauss ss, [7] divb ss
    unsigned long long* amax = reinterpret_cast<unsigned long long*>(g->diag_acc + 8);   // [0] divB, [1] gauss
    HYB_CUDA_TRY(cudaMemsetAsync(g->diag_acc, 0, 16 * sizeof(double), g->stream));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const unsigned blocks = (unsigned)(sms * 4);

    Ptr6 f6{};
    for (int c = 0; c < 3; c++) { f6.p[c] = g->E[c]; f6.p[3 + c] = g->B[c]; }
    k_energy<T><<<dim3(blocks, 6), kDiagThreads, 0, g->stream>>>(f6, cells, acc);
    HYB_CUDA_TRY(cudaGetLastError());

    const double inv2 = 1.0 / d.dx2, inv3 = d.dims == 3 ? 1.0 / d.dx3 : 0.0;
    // div B
    HYB_CUDA_TRY((rfft_rows<T, double>((const T*)g->B[0], s1, n1, rows, g->td, g->stream)));
    k_mul_sigma<<<(unsigned)rows, kDiagThreads, 0, g->stream>>>(s1, nk, rows, g->td.sgp, +1);
    HYB_CUDA_TRY(cudaGetLastError());
    HYB_CUDA_TRY((irfft_rows<double, double>(s1, D, n1, rows, g->td, g->stream)));
    k_add_fd<T><<<blocks, kDiagThreads, 0, g->stream>>>(D, (const T*)g->B[1], d.dims == 3 ? (const T*)g->B[2] : nullptr,
                                                        n1, d.n2, n3, inv2, inv3, 1, acc + 7, amax + 0);
    HYB_CUDA_TRY(cudaGetLastError());
    // Gauss residual
    HYB_CUDA_TRY((rfft_rows<T, double>((const T*)g->E[0], s1, n1, rows, g->td, g->stream)));
    k_mul_sigma<<<(unsigned)rows, kDiagThreads, 0, g->stream>>>(s1, nk, rows, g->td.sgp, -1);
    HYB_CUDA_TRY(cudaGetLastError());
    if (g->rho) {
        HYB_CUDA_TRY((rfft_rows<T, double>((const T*)g->rho, s2, n1, rows, g->td, g->stream)));
        k_sub_filtered<<<(unsigned)rows, kDiagThreads, 0, g->stream>>>(s1, s2, nk, rows, g->td.filt, d.ampere);
        HYB_CUDA_TRY(cudaGetLastError());
    }
    HYB_CUDA_TRY((irfft_rows<double, double>(s1, D, n1, rows, g->td, g->stream)));
    k_add_fd<T><<<blocks, kDiagThreads, 0, g->stream>>>(D, (const T*)g->E[1], d.dims == 3 ? (const T*)g->E[2] : nullptr,
                                                        n1, d.n2, n3, inv2, inv3, 0, acc + 6, amax + 1);
    HYB_CUDA_TRY(cudaGetLastError());
    double h[16];
    HYB_CUDA_TRY(cudaMemcpyAsync(h, g->diag_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(g->stream));
    const double dV = d.dx1 * d.dx2 * (d.dims == 3 ? d.dx3 : 1.0);
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < 6; c++) out[c] = h[c] * dV / (8.0 * pi);
    unsigned long long km[2];
    memcpy(km, &h[8], sizeof(km));
    double mx[2];
    memcpy(&mx[0], &km[0], sizeof(double));
    memcpy(&mx[1], &km[1], sizeof(double));
    out[6] = mx[0];
    out[7] = mx[1];
    out[8] = sqrt(h[6] / (double)cells);
    return HYB_OK;
}

template hyb_status diag<float>(hyb_grid*, double[9]);
template hyb_status diag<double>(hyb_grid*, double[9]);

}  // namespace hyb
