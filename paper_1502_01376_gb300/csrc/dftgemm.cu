// dftgemm.cu -- the x1 transform of the three-pass advance as a dense DFT
// matrix product on the tensor cores (path 3), for short n1.  FP32 operands
// are split into two BF16 parts, a = a_hi + a_lo, and the product keeps the
// three leading terms a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32
// (mma.sync m16n8k16): one GEMM with the K dimension tripled,
//   [a_hi | a_hi | a_lo] x [b_hi ; b_lo ; b_hi].
// Forward:  X[r][2k + {0,1}] = sum_j x[r][j] (cos, -sin)(2 pi k j / n1), k = 0..n1/2
// Inverse:  x[r][j] = sum_k w_k (Re X_k cos - Im X_k sin)(2 pi k j / n1) / n1,
//           w_0 = w_{n1/2} = 1, otherwise 2 (the imaginary parts of the DC and
//           Nyquist coefficients drop out, as in the radix path).
// The matrices are computed in FP64 on the host and split once.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "hyb_internal.cuh"

namespace hyb {

constexpr int GM = 64, GN = 64, GK = 16;

__device__ __forceinline__ uint32_t pk2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// C[m][n] (FP32, row stride ldc) = sum_k A[m][k] B[k][n]; A BF16 row-major (lda),
// B BF16 row-major (ldb); K multiple of 16; M, N arbitrary.
__global__ void __launch_bounds__(128) k_dgemm(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int64_t lda,
                                               const __nv_bfloat16* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                               int64_t ldc) {
    __shared__ __nv_bfloat16 As[GM][GK + 8];
    __shared__ __nv_bfloat16 Bs[GN][GK + 8];
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int i = threadIdx.x; i < GM * GK; i += blockDim.x) {
            const int r = i / GK, kk = i % GK, m = m0 + r;
            As[r][kk] = (m < M) ? A[(int64_t)m * lda + k0 + kk] : __float2bfloat16(0.f);
        }
        for (int i = threadIdx.x; i < GN * GK; i += blockDim.x) {
            const int kk = i / GN, r = i % GN, n = n0 + r;
            Bs[r][kk] = (n < N) ? B[(int64_t)(k0 + kk) * ldb + n] : __float2bfloat16(0.f);
        }
        __syncthreads();
        uint32_t af[2][4], bf[4][2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int r = wm + i * 16;
            af[i][0] = pk2(As[r + gq][2 * tq], As[r + gq][2 * tq + 1]);
            af[i][1] = pk2(As[r + gq + 8][2 * tq], As[r + gq + 8][2 * tq + 1]);
            af[i][2] = pk2(As[r + gq][2 * tq + 8], As[r + gq][2 * tq + 9]);
            af[i][3] = pk2(As[r + gq + 8][2 * tq + 8], As[r + gq + 8][2 * tq + 9]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int cn = wn + j * 8 + gq;
            bf[j][0] = pk2(Bs[cn][2 * tq], Bs[cn][2 * tq + 1]);
            bf[j][1] = pk2(Bs[cn][2 * tq + 8], Bs[cn][2 * tq + 9]);
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                             "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                             : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                             : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = m0 + wm + i * 16 + gq + 8 * h, cc = n0 + wn + j * 8 + 2 * tq;
                if (r < M) {
                    if (cc < N) C[(int64_t)r * ldc + cc] = acc[i][j][2 * h];
                    if (cc + 1 < N) C[(int64_t)r * ldc + cc + 1] = acc[i][j][2 * h + 1];
                }
            }
}

struct SplitSrc { const float* p[9]; };

// rows of the nf source arrays (row length L, row stride ls) -> BF16 [nf*rows][3 Lp]:
// [hi | hi | lo], each segment padded with zeros to Lp (a multiple of 16)
__global__ void k_split_rows(SplitSrc src, int nf, int64_t rows, int L, int Lp, int64_t ls, __nv_bfloat16* __restrict__ out) {
    const int64_t R = (int64_t)nf * rows;
    const int64_t total = R * Lp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / Lp;
        const int c = (int)(i % Lp);
        const int f = (int)(r / rows);
        const float v = (c < L) ? src.p[f][(r % rows) * ls + c] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16(v);
        const __nv_bfloat16 lo = __float2bfloat16(v - __bfloat162float(hi));
        __nv_bfloat16* o = out + r * (3 * (int64_t)Lp);
        o[c] = hi;
        o[Lp + c] = hi;
        o[2 * Lp + c] = lo;
    }
}

struct DftPlan {
    __nv_bfloat16* Bf = nullptr;   // [3 n1][n1 + 2]
    __nv_bfloat16* Bi = nullptr;   // [3 (n1 + 2)][n1]
    __nv_bfloat16* Asplit = nullptr;
    size_t a_elems = 0;
};

static void split_host(const std::vector<double>& m, std::vector<__nv_bfloat16>& hi, std::vector<__nv_bfloat16>& lo) {
    hi.resize(m.size());
    lo.resize(m.size());
    for (size_t i = 0; i < m.size(); i++) {
        const float f = (float)m[i];
        hi[i] = __float2bfloat16(f);
        lo[i] = __float2bfloat16(f - __bfloat162float(hi[i]));
    }
}

hyb_status dftgemm_create(hyb_grid* g) {
    const int n = g->d.n1, nc = n + 2;
    const double pi = 3.14159265358979323846;
    std::vector<double> F((size_t)n * nc), I((size_t)nc * n);
    for (int j = 0; j < n; j++)
        for (int k = 0; k <= n / 2; k++) {
            const double a = 2.0 * pi * (double)(((int64_t)k * j) % n) / n;
            F[(size_t)j * nc + 2 * k] = cos(a);
            F[(size_t)j * nc + 2 * k + 1] = -sin(a);
            const double w = (k == 0 || k == n / 2) ? 1.0 : 2.0;
            I[(size_t)(2 * k) * n + j] = w * cos(a) / n;
            I[(size_t)(2 * k + 1) * n + j] = -w * sin(a) / n;
        }
    const int ncp = (nc + 15) & ~15;          // inverse K segment, padded with zero rows
    I.resize((size_t)ncp * n, 0.0);
    std::vector<__nv_bfloat16> fh, fl, ih, il;
    split_host(F, fh, fl);
    split_host(I, ih, il);
    // stacked [hi; lo; hi] along K
    std::vector<__nv_bfloat16> Bf((size_t)3 * n * nc), Bi((size_t)3 * ncp * n);
    for (size_t i = 0; i < fh.size(); i++) { Bf[i] = fh[i]; Bf[fh.size() + i] = fl[i]; Bf[2 * fh.size() + i] = fh[i]; }
    for (size_t i = 0; i < ih.size(); i++) { Bi[i] = ih[i]; Bi[ih.size() + i] = il[i]; Bi[2 * ih.size() + i] = ih[i]; }
    DftPlan* P = new DftPlan();
    g->dft = P;
    HYB_CUDA_TRY(cudaMalloc(&P->Bf, sizeof(__nv_bfloat16) * Bf.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->Bf, Bf.data(), sizeof(__nv_bfloat16) * Bf.size(), cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMalloc(&P->Bi, sizeof(__nv_bfloat16) * Bi.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->Bi, Bi.data(), sizeof(__nv_bfloat16) * Bi.size(), cudaMemcpyHostToDevice));
    P->a_elems = (size_t)9 * g->rows * 3 * ncp;
    HYB_CUDA_TRY(cudaMalloc(&P->Asplit, sizeof(__nv_bfloat16) * P->a_elems));
    return HYB_OK;
}

void dftgemm_destroy(hyb_grid* g) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    if (!P) return;
    cudaFree(P->Bf); cudaFree(P->Bi); cudaFree(P->Asplit);
    delete P;
    g->dft = nullptr;
}

static void dgemm(int M, int N, int K, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, float* C,
                  int64_t ldc, cudaStream_t s) {
    dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN);     // M tiles on x: up to 2^31 - 1 blocks
    k_dgemm<<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

// forward transform of nf fields into spec (FP32 complex [nf][rows][n1/2+1])
hyb_status dftgemm_forward(hyb_grid* g, const float* const* fields, int nf, float2* spec) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    const int n = g->d.n1, nc = n + 2;
    const int64_t rows = g->rows;
    SplitSrc src{};
    for (int f = 0; f < nf; f++) src.p[f] = fields[f];
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    k_split_rows<<<sms * 8, 256, 0, g->stream>>>(src, nf, rows, n, n, n, P->Asplit);
    HYB_CUDA_TRY(cudaGetLastError());
    dgemm((int)(nf * rows), nc, 3 * n, P->Asplit, 3 * n, P->Bf, nc, reinterpret_cast<float*>(spec), nc, g->stream);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

// inverse transform of the first nf spectral fields back into the real fields
hyb_status dftgemm_inverse(hyb_grid* g, const float2* spec, int nf, float* const* fields) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    const int n = g->d.n1, nc = n + 2;
    const int64_t rows = g->rows;
    SplitSrc src{};
    for (int f = 0; f < nf; f++) src.p[f] = reinterpret_cast<const float*>(spec) + (size_t)f * rows * nc;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int ncp = (nc + 15) & ~15;
    k_split_rows<<<sms * 8, 256, 0, g->stream>>>(src, nf, rows, nc, ncp, nc, P->Asplit);
    HYB_CUDA_TRY(cudaGetLastError());
    // one product per field, written straight into its array
    for (int f = 0; f < nf; f++)
        dgemm((int)rows, n, 3 * ncp, P->Asplit + (size_t)f * rows * 3 * ncp, 3 * ncp, P->Bi, n, fields[f], n, g->stream);
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

}  // namespace hyb
