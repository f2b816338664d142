// dftgemm.cu -- the x1 transform of the three-pass advance as a dense DFT
// matrix product on the fifth-generation tensor cores (path 3), for short n1.
//
// Forward:  X[r][2k + {0,1}] = sum_j x[r][j] (cos, -sin)(2 pi k j / n1), k = 0..n1/2
// Inverse:  x[r][j] = sum_k w_k (Re X_k cos - Im X_k sin)(2 pi k j / n1) / n1,
//           w_0 = w_{n1/2} = 1, otherwise 2 (the imaginary parts of the DC and
//           Nyquist coefficients drop out, as in the radix path).
// Both are D[m][n] = sum_k A[m][k] M[n][k] with A the FP32 rows (K = n1 reals,
// or n1 + 2 interleaved spectrum values) and M the DFT matrix, computed in FP64
// on the host and rounded to FP32.  FP32 operands are split into two BF16
// parts, a = a_hi + a_lo, and the product keeps the three leading terms
//   D = A_hi M_hi + A_hi M_lo + A_lo M_hi,
// accumulated in FP32 by tcgen05.mma (kind::f16, BF16 inputs) in tensor memory.
//
// k_dft_tc: a persistent kernel over (tile of 128 rows, pass of <= 512 output
// columns).  Per 64-wide K chunk the 256 threads load the tile's FP32 values
// (coalesced along the rows), split them and store A_hi, A_lo in shared memory
// in the canonical K-major layout without swizzle (core matrices of 8 rows x
// 16 bytes; element (m, k) at byte (k / 8) * LBO + 16 m + 2 (k % 8)); the
// matrix chunk, stored in global memory in that layout already, arrives by one
// bulk copy (cp.async.bulk, completion on an mbarrier).  One thread issues the
// 4 k-steps x 3 products x (1 or 2 column blocks of <= 256) MMAs into the TMEM
// accumulator (row m in lane m, column n in column n) and commits them to a
// second mbarrier; the next chunk overwrites shared memory only after it.  The
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w % 4) ..,
// half of the column blocks) and writes the valid columns of each row.  All
// waits are bounded; a wait that runs out sets bit 1 of the grid's error flag,
// skips the remaining work, drains what is in flight and frees the TMEM.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "hyb_internal.cuh"
#include "tm_dev.cuh"

namespace hyb {

namespace dg {
constexpr int BM = 128;                  // rows per tile (MMA M)
constexpr int KC = 64;                   // K per chunk: 4 k-steps of 16
constexpr int NPASS = 512;               // output columns per pass (TMEM columns)
constexpr int NT = 256;                  // threads per CTA
constexpr int A_LBO = BM * 16 + 32;      // bytes between K groups of the A image (padded: bank spread)
constexpr int A_IMG = 8 * A_LBO;         // one A image (hi or lo) of a chunk
constexpr int OFF_B = ((2 * A_IMG + 127) / 128) * 128;
// shared memory requested beyond the operand images, so that the products of a chunk stay
// inside the CTA's allocation whichever of the two byte offsets of the descriptor the
// hardware applies along K (the images are laid out for the K-direction one)
constexpr int GUARD = 0;
}  // namespace dg

// shared-memory matrix descriptor of tcgen05: start, leading (K-direction core matrix) and
// stride (M/N-direction 8-row group) byte offsets, fixed version bits 46-48 = 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}
// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}
// bounded wait that ignores the abort flag: used to drain copies and products in flight
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

struct DgArgs {
    const float* src[9];          // source arrays: rows x L valid values, row stride ls floats
    float* dst[9];                // destination arrays: rows x N valid values, row stride ld floats
    int nf;
    int64_t rows;                 // rows per array
    int L, ls;
    int N, ld;
    int nkc;                      // K chunks of 64
    int npass;                    // passes over the output columns
    int npc[4];                   // columns of pass p (multiple of 16, <= 512)
    int64_t boff[4];              // element offset of pass p's first chunk image in B
    const __nv_bfloat16* B;       // per (pass, chunk): hi image then lo image, each npc x 64
    uint32_t tcols;               // TMEM columns allocated
    int* err;
};

// P value pairs per row and warp row (P = 32, or 16 / 8 when a row has at most 32 / 16 values):
// thread tid loads, for (tile, chunk kc), rows tid / P + (256 / P) j of the tile (j < P / 2),
// values kc * 64 + 2 (tid % P) and the next; zero outside the arrays
template <int P>
__device__ __forceinline__ void dg_load(const DgArgs& a, int64_t tile, int kc, int tid, float2 (&v)[16]) {
    const int64_t t0 = tile * dg::BM;
    const int f0 = (int)(t0 / a.rows);
    const int64_t r0 = t0 - (int64_t)f0 * a.rows;
    const int k = kc * dg::KC + 2 * (tid % P);
#pragma unroll
    for (int j = 0; j < P / 2; j++) {
        int f = f0;
        int64_t r = r0 + tid / P + (dg::NT / P) * j;
        while (r >= a.rows) { r -= a.rows; f++; }
        v[j] = make_float2(0.f, 0.f);
        if (f < a.nf && k < a.L) {
            const float* row = a.src[f] + r * a.ls;
            if (k + 1 < a.L) v[j] = __ldg(reinterpret_cast<const float2*>(row + k));
            else v[j].x = __ldg(row + k);
        }
    }
}
// the same pairs split into BF16 hi and lo parts, stored into the two A images
template <int P>
__device__ __forceinline__ void dg_store(uint32_t sA, int tid, const float2 (&v)[16]) {
    const int kk = 2 * (tid % P);
#pragma unroll
    for (int j = 0; j < P / 2; j++) {
        const int i = tid / P + (dg::NT / P) * j;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[j].x), h1 = __float2bfloat16_rn(v[j].y);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[j].x - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[j].y - __bfloat162float(h1));
        const uint32_t off = (uint32_t)((kk >> 3) * dg::A_LBO + 16 * i + 2 * (kk & 7));
        const uint32_t hv = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        const uint32_t lv = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        asm volatile("st.shared.b32 [%0], %1;" :: "r"(sA + off), "r"(hv) : "memory");
        asm volatile("st.shared.b32 [%0], %1;" :: "r"(sA + dg::A_IMG + off), "r"(lv) : "memory");
    }
}

template <int P>
__global__ void __launch_bounds__(dg::NT, 1) k_dft_tc(DgArgs a) {
    using namespace dg;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t bars[2];                 // 0: matrix chunk landed, 1: products done
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sA = (smem_addr(sm) + 127u) & ~127u;          // 128 bytes of slack are requested
    const uint32_t sB = sA + OFF_B;
    const uint32_t bar_b = smem_addr(&bars[0]), bar_m = smem_addr(&bars[1]);
    if (warp == 0) {
        tm_alloc(smem_addr(&s_taddr), a.tcols);
        tm_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_b, 1);
        mbar_init(bar_m, 1);
        mbar_fence_init();
        s_abort = 0;
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = s_taddr;
    uint32_t ph_b = 0, ph_m = 0;
    bool pend_b = false, pend_m = false;         // thread 0: a copy / products not yet waited for
    bool b_in = false;                           // thread 0: the single matrix image is in shared memory
    const bool b_resident = a.nkc * a.npass == 1;
    const int64_t R = (int64_t)a.nf * a.rows;
    const int64_t items = (R + BM - 1) / BM * a.npass;
    bool abort = false;                          // s_abort as read after a barrier: uniform
    // units (item, chunk) of this CTA in order; the values of the next unit are loaded while the
    // products of the current one run
    int64_t it = blockIdx.x;
    int kc = 0;
    float2 v[16];
    if (it < items) dg_load<P>(a, it / a.npass, 0, tid, v);
    while (it < items && !abort) {
        const int64_t tile = it / a.npass;
        const int p = (int)(it % a.npass);
        const int npc = a.npc[p];
        const int c0 = npc < 256 ? npc : 256, c1 = npc - c0;
        if (tid == 0 && !(b_resident && b_in)) {
            const uint32_t bytes = (uint32_t)npc * KC * 2 * 2;
            mbar_expect_tx(bar_b, bytes);
            bulk_load(sB, a.B + a.boff[p] + (int64_t)kc * 2 * npc * KC, bytes, bar_b);
            pend_b = true;
        }
        dg_store<P>(sA, tid, v);
        fence_proxy_async_smem();
        tm_fence_before();
        __syncthreads();
        if (tid == 0) {
            tm_fence_after();
            if (pend_b) {
                mbar_wait(bar_b, ph_b, a.err, &s_abort);
                if (!s_abort) {
                    ph_b ^= 1;
                    pend_b = false;
                    b_in = true;
                }
            }
            if (!s_abort) {
                // k-steps of 16 holding values of this chunk (the rest of the image is zero)
                const int nks = min(4, (a.L - kc * KC + 15) / 16);
                for (int ks = 0; ks < nks; ks++) {
                    const uint64_t ah = smem_desc(sA + 2 * ks * A_LBO, A_LBO, 128);
                    const uint64_t al = smem_desc(sA + A_IMG + 2 * ks * A_LBO, A_LBO, 128);
                    for (int c = 0; c < 2; c++) {
                        const int w = c ? c1 : c0;
                        if (w == 0) continue;
                        // the block's hi and lo images: 8 K groups of w rows x 16 bytes each
                        const uint32_t bh = sB + (uint32_t)(c ? c0 : 0) * KC * 2;
                        const uint32_t bl = bh + (uint32_t)npc * KC * 2;
                        const uint32_t lb = (uint32_t)w * 16;
                        const uint64_t dh = smem_desc(bh + 2 * ks * lb, lb, 128);
                        const uint64_t dl = smem_desc(bl + 2 * ks * lb, lb, 128);
                        const uint32_t dt = tbase + (uint32_t)(c ? c0 : 0);
                        const uint32_t id = idesc_bf16(w);
                        mma_bf16(dt, ah, dh, id, (kc > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(dt, ah, dl, id, 1u);
                        mma_bf16(dt, al, dh, id, 1u);
                    }
                }
                mma_commit(bar_m);
                pend_m = true;
            }
        }
        // the next unit's values, in flight while the products run
        int64_t it2 = it;
        int kc2 = kc + 1;
        if (kc2 == a.nkc) { it2 = it + gridDim.x; kc2 = 0; }
        if (it2 < items) dg_load<P>(a, it2 / a.npass, kc2, tid, v);
        if (tid == 0 && pend_m) {
            // the products read shared memory: wait for them before the next unit overwrites it
            mbar_wait(bar_m, ph_m, a.err, &s_abort);
            if (!s_abort) {
                ph_m ^= 1;
                pend_m = false;
            }
        }
        __syncthreads();
        abort = s_abort != 0;
        if (kc == a.nkc - 1 && !abort) {
            // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows), column units of 16
            // alternating between the two warp halves
            tm_fence_after();
            const int q = warp & 3, h = warp >> 2;
            int f = 0;
            int64_t r = 0;
            {
                const int64_t gr = tile * BM + 32 * q + lane;
                f = (int)(gr / a.rows);
                r = gr - (int64_t)f * a.rows;
            }
            float* out = f < a.nf ? a.dst[f] + r * a.ld : nullptr;
            for (int u = h; u < npc / 16; u += 2) {
                float t[16];
                tm_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * u), t);
                tm_wait_ld();
                const int n0 = p * NPASS + 16 * u;
                if (out) {
#pragma unroll
                    for (int j = 0; j < 16; j += 2)
                        if (n0 + j < a.N) *reinterpret_cast<float2*>(out + n0 + j) = make_float2(t[j], t[j + 1]);
                }
            }
            tm_fence_before();
        }
        it = it2;
        kc = kc2;
    }
    // drain what an early exit left in flight, then free the tensor memory
    if (tid == 0) {
        if (pend_b) mbar_drain(bar_b, ph_b);
        if (pend_m) mbar_drain(bar_m, ph_m);
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, a.tcols);
}

// ------------------------------------------------------------------ host side
struct DftOp {                      // one direction: matrix images and launch shape
    __nv_bfloat16* B = nullptr;
    int K = 0, N = 0, nkc = 0, npass = 0;
    int npc[4] = {0, 0, 0, 0};
    int64_t boff[4] = {0, 0, 0, 0};
    uint32_t tcols = 0;
    size_t smem = 0;
    int grid = 0;
    void (*kern)(DgArgs) = nullptr;     // k_dft_tc<P>, P = pairs per row and warp row
};
struct DftPlan {
    DftOp fwd, inv;
};

// M[n][k] (FP64, n < N, k < K) -> images [pass][chunk][hi | lo][block][k / 8][n][k % 8] of BF16
static hyb_status make_op(hyb_grid* g, DftOp& op, const std::vector<double>& M, int N, int K) {
    using namespace dg;
    op.K = K;
    op.N = N;
    op.nkc = (K + KC - 1) / KC;
    const int Np = (N + 15) & ~15;
    op.npass = (Np + NPASS - 1) / NPASS;
    if (op.npass > 4) { set_error("DFT-GEMM: n1 too large"); return HYB_EINVAL; }
    size_t total = 0;
    int maxc = 0;
    for (int p = 0; p < op.npass; p++) {
        op.npc[p] = std::min(NPASS, Np - p * NPASS);
        op.boff[p] = (int64_t)total;
        total += (size_t)op.nkc * 2 * op.npc[p] * KC;
        maxc = std::max(maxc, op.npc[p]);
    }
    std::vector<__nv_bfloat16> img(total, __float2bfloat16(0.f));
    for (int p = 0; p < op.npass; p++) {
        const int npc = op.npc[p];
        const int c0 = std::min(256, npc);
        for (int kc = 0; kc < op.nkc; kc++) {
            __nv_bfloat16* base = img.data() + op.boff[p] + (size_t)kc * 2 * npc * KC;
            for (int nl = 0; nl < npc; nl++) {
                const int blk = nl < c0 ? 0 : 1, w = blk ? npc - c0 : c0, nb = blk ? nl - c0 : nl;
                const size_t boff = (size_t)(blk ? c0 : 0) * KC;
                for (int kl = 0; kl < KC; kl++) {
                    const int n = p * NPASS + nl, k = kc * KC + kl;
                    const float v = (n < N && k < K) ? (float)M[(size_t)n * K + k] : 0.f;
                    const __nv_bfloat16 hi = __float2bfloat16(v);
                    const __nv_bfloat16 lo = __float2bfloat16(v - __bfloat162float(hi));
                    const size_t e = boff + ((size_t)(kl >> 3) * w + nb) * 8 + (kl & 7);
                    base[e] = hi;
                    base[(size_t)npc * KC + e] = lo;
                }
            }
        }
    }
    HYB_CUDA_TRY(cudaMalloc(&op.B, sizeof(__nv_bfloat16) * total));
    HYB_CUDA_TRY(cudaMemcpy(op.B, img.data(), sizeof(__nv_bfloat16) * total, cudaMemcpyHostToDevice));
    op.tcols = maxc <= 256 ? 256 : 512;
    op.smem = 128 + (size_t)OFF_B + (size_t)maxc * KC * 2 * 2 + GUARD;
    op.kern = K <= 16 ? k_dft_tc<8> : K <= 32 ? k_dft_tc<16> : k_dft_tc<32>;
    const void* kf = (const void*)op.kern;
    HYB_CUDA_TRY(func_attr_once(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(128 + OFF_B + NPASS * KC * 2 * 2 + GUARD)));
    HYB_CUDA_TRY(func_attr_once(kf, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // CTAs per SM from the kernel's registers and shared memory (warps take registers in units
    // of 256) and from the 512 TMEM columns the CTAs of an SM share
    cudaFuncAttributes fa;
    HYB_CUDA_TRY(cudaFuncGetAttributes(&fa, kf));
    int sms = 0, smem_sm = 0;
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, g->device));
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int occ_r = 65536 / (regs_warp * (NT / 32));
    const int occ_s = (int)(smem_sm / (op.smem + fa.sharedSizeBytes + 1024));
    const int occ = std::max(1, std::min({occ_r, occ_s, (int)(512 / op.tcols)}));
    op.grid = sms * occ;
    return HYB_OK;
}

hyb_status dftgemm_create(hyb_grid* g) {
    const int n = g->d.n1, nc = n + 2;
    const double pi = 3.14159265358979323846;
    std::vector<double> F((size_t)nc * n), I((size_t)n * nc);     // F[out][in], I[out][in]
    for (int j = 0; j < n; j++)
        for (int k = 0; k <= n / 2; k++) {
            const double ang = 2.0 * pi * (double)(((int64_t)k * j) % n) / n;
            F[(size_t)(2 * k) * n + j] = cos(ang);
            F[(size_t)(2 * k + 1) * n + j] = -sin(ang);
            const double w = (k == 0 || k == n / 2) ? 1.0 : 2.0;
            I[(size_t)j * nc + 2 * k] = w * cos(ang) / n;
            I[(size_t)j * nc + 2 * k + 1] = -w * sin(ang) / n;
        }
    DftPlan* P = new DftPlan();
    g->dft = P;
    hyb_status st = make_op(g, P->fwd, F, nc, n);
    if (st == HYB_OK) st = make_op(g, P->inv, I, n, nc);
    return st;
}

void dftgemm_destroy(hyb_grid* g) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    if (!P) return;
    cudaFree(P->fwd.B);
    cudaFree(P->inv.B);
    delete P;
    g->dft = nullptr;
}

static cudaError_t launch_op(const hyb_grid* g, const DftOp& op, const float* const* src, int ls, float* const* dst,
                             int ld, int nf) {
    DgArgs a{};
    for (int f = 0; f < nf; f++) { a.src[f] = src[f]; a.dst[f] = dst[f]; }
    a.nf = nf;
    a.rows = g->rows;
    a.L = op.K;
    a.ls = ls;
    a.N = op.N;
    a.ld = ld;
    a.nkc = op.nkc;
    a.npass = op.npass;
    for (int p = 0; p < 4; p++) { a.npc[p] = op.npc[p]; a.boff[p] = op.boff[p]; }
    a.B = op.B;
    a.tcols = op.tcols;
    a.err = g->dflag;
    const int64_t items = ((int64_t)nf * g->rows + dg::BM - 1) / dg::BM * op.npass;
    const int grid = (int)std::min<int64_t>(op.grid, items);
    op.kern<<<grid, dg::NT, op.smem, g->stream>>>(a);
    return cudaGetLastError();
}

// forward transform of nf fields into spec (FP32 complex [nf][rows][n1/2+1])
hyb_status dftgemm_forward(hyb_grid* g, const float* const* fields, int nf, float2* spec) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    const int n = g->d.n1, nc = n + 2;
    float* dst[9];
    for (int f = 0; f < nf; f++) dst[f] = reinterpret_cast<float*>(spec) + (size_t)f * g->rows * nc;
    HYB_CUDA_TRY(launch_op(g, P->fwd, fields, n, dst, nc, nf));
    return HYB_OK;
}

// inverse transform of the first nf spectral fields back into the real fields
hyb_status dftgemm_inverse(hyb_grid* g, const float2* spec, int nf, float* const* fields) {
    DftPlan* P = reinterpret_cast<DftPlan*>(g->dft);
    const int n = g->d.n1, nc = n + 2;
    const float* src[9];
    for (int f = 0; f < nf; f++) src[f] = reinterpret_cast<const float*>(spec) + (size_t)f * g->rows * nc;
    HYB_CUDA_TRY(launch_op(g, P->inv, src, nc, const_cast<float* const*>(fields), n, nf));
    return HYB_OK;
}

}  // namespace hyb
