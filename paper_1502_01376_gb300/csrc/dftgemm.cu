// dftgemm.cu -- the x1 transform of the three-pass advance as a dense DFT
// matrix product on the fifth-generation tensor cores (path 3), for short n1.
//
// Forward:  X[r][2k + {0,1}] = sum_j x[r][j] (cos, -sin)(2 pi k j / n1), k = 0..n1/2
// Inverse:  x[r][j] = sum_k w_k (Re X_k cos - Im X_k sin)(2 pi k j / n1) / n1,
//           w_0 = w_{n1/2} = 1, otherwise 2 (the imaginary parts of the DC and
//           Nyquist coefficients drop out, as in the radix path).
// Both are D[m][n] = sum_k A[m][k] M[n][k] with A the FP32 rows (K = n1 reals,
// or n1 + 2 interleaved spectrum values) and M the DFT matrix, computed in FP64
// on the host and rounded to FP32.  FP32 operands are split into S BF16 parts,
// a = a_0 + a_1 (+ a_2), a_{i+1} the BF16 rounding of what a_0 .. a_i leave,
// and the product keeps the terms A_i M_j with i + j < S:
//   S = 2 (path 3): A_0 M_0 + A_0 M_1 + A_1 M_0              (three products)
//   S = 3 (path 4): the same + A_0 M_2 + A_1 M_1 + A_2 M_0   (six products)
// accumulated in FP32 by tcgen05.mma (kind::f16, BF16 inputs) in tensor memory.
// The dropped terms and the last part's rounding leave about 2^-17 (S = 2) or
// 2^-25 (S = 3) relative error per product term.
//
// k_dft_tc: a persistent kernel over (tile of 128 rows, pass of <= 512 (S = 2)
// or 256 (S = 3) output columns).  Per 64-wide K chunk the 256 threads load the
// tile's FP32 values (coalesced along the rows), split them and store the S
// parts A_i in shared memory
// in the canonical K-major layout without swizzle (core matrices of 8 rows x
// 16 bytes; element (m, k) at byte (k / 8) * LBO + 16 m + 2 (k % 8)); the
// matrix chunk, stored in global memory in that layout already, arrives by one
// bulk copy (cp.async.bulk, completion on an mbarrier).  One thread issues the
// k-steps x products x (1 or 2 column blocks of <= 256) MMAs into the TMEM
// accumulator (row m in lane m, column n in column n) and commits them to a
// second mbarrier; the next chunk overwrites shared memory only after it.  The
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w % 4) ..,
// half of the column blocks); where the tile's output rows are contiguous it
// stages them in shared memory (64 or 32 rows per round, the A images being
// free then) and copies each block out in order, else it stores each row.  The
// imaginary parts of the DC and Nyquist coefficients are zero, so the forward
// product computes the Nyquist real part in column 1 (n1 product columns for
// n1 + 2 outputs) and the inverse reads it in that slot (K = n1).  All
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
constexpr int MAXPASS = 8;               // passes over the output columns (n1 <= 1024)
constexpr int NT = 256;                  // threads per CTA
// bytes between K groups of the A image: 2048 plus a pad that puts the 8 K groups of a row 4
// banks apart (A_LBO / 4 = 4 mod 32), so a warp's split stores hit 32 banks; the two images
// together also hold the 64 x 130 FP32 staging block of the epilogue
constexpr int A_LBO = BM * 16 + 144;
constexpr int A_IMG = 8 * A_LBO;         // one A image (one part) of a chunk
__host__ __device__ constexpr int off_b(int S) { return ((S * A_IMG + 127) / 128) * 128; }
__host__ __device__ constexpr int pass_cols(int S) { return S == 2 ? 512 : 256; }
}  // namespace dg

struct DgArgs {
    const float* src[9];          // source arrays: rows x L valid values, row stride ls floats
    float* dst[9];                // destination arrays: rows x N valid values, row stride ld floats
    int nf;
    int64_t rows;                 // rows per array
    int L, ls;                    // K extent of the product, source row stride
    int N, ld;                    // output columns written, destination row stride
    // 1: the K slot 1 (the DC imaginary part, whose coefficients are zero) carries the value at
    //    position L (the Nyquist real part): K = n1 instead of n1 + 2 (inverse);
    // 2: product column 1 is the Nyquist real part, written to column N - 2, with columns 1 and
    //    N - 1 (the zero imaginary parts of DC and Nyquist) set to 0 (forward)
    int fold;
    int nkc;                      // K chunks of 64
    int npass;                    // passes over the output columns
    int npc[dg::MAXPASS];         // columns of pass p (multiple of 16, <= pass_cols(S))
    int64_t boff[dg::MAXPASS];    // element offset of pass p's first chunk image in B
    const __nv_bfloat16* B;       // per (pass, chunk): the S part images, each npc x 64
    uint32_t tcols;               // TMEM columns allocated
    int* err;
};

// P value pairs per row and warp row (P = 32, or 16 / 8 when a row has at most 32 / 16 values):
// thread tid loads, for (tile, chunk kc), rows tid / P + (256 / P) j of the tile (j < P / 2),
// values kc * 64 + 2 (tid % P) and the next; zero outside the arrays
template <int P, bool FIN>
__device__ __forceinline__ void dg_load(const DgArgs& a, int64_t tile, int kc, int tid, float2 (&v)[16], float (&vn)[16]) {
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
            // the Nyquist real part for the DC imaginary slot, in its own register: no load waits
            // on another one before the values are stored
            if (FIN && k == 0) vn[j] = __ldg(row + a.L);
        }
    }
}
// the same pairs split into S BF16 parts (each the rounding of what the earlier parts leave;
// the differences are exact in FP32), stored into the S A images
template <int P, int S, bool FIN>
__device__ __forceinline__ void dg_store(uint32_t sA, int tid, int kc, const float2 (&v)[16], const float (&vn)[16]) {
    const int kk = 2 * (tid % P);
#pragma unroll
    for (int j = 0; j < P / 2; j++) {
        const int i = tid / P + (dg::NT / P) * j;
        const uint32_t off = (uint32_t)((kk >> 3) * dg::A_LBO + 16 * i + 2 * (kk & 7));
        float r0 = v[j].x, r1 = (FIN && kc == 0 && kk == 0) ? vn[j] : v[j].y;
#pragma unroll
        for (int q = 0; q < S; q++) {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(r0), b1 = __float2bfloat16_rn(r1);
            r0 -= __bfloat162float(b0);
            r1 -= __bfloat162float(b1);
            const uint32_t w = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
            asm volatile("st.shared.b32 [%0], %1;" :: "r"(sA + q * dg::A_IMG + off), "r"(w) : "memory");
        }
    }
}

template <int P, int S, bool FIN>
__global__ void __launch_bounds__(dg::NT, 2) k_dft_tc(DgArgs a) {
    using namespace dg;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t bars[2];                 // 0: matrix chunk landed, 1: products done
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sA = (smem_addr(sm) + 127u) & ~127u;          // 128 bytes of slack are requested
    const uint32_t sB = sA + off_b(S);
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
    float vn[16];
    if (it < items) dg_load<P, FIN>(a, it / a.npass, 0, tid, v, vn);
    while (it < items && !abort) {
        const int64_t tile = it / a.npass;
        const int p = (int)(it % a.npass);
        const int npc = a.npc[p];
        const int c0 = npc < 256 ? npc : 256, c1 = npc - c0;
        if (tid == 0 && !(b_resident && b_in)) {
            const uint32_t bytes = (uint32_t)npc * KC * 2 * S;
            mbar_expect_tx(bar_b, bytes);
            bulk_load(sB, a.B + a.boff[p] + (int64_t)kc * S * npc * KC, bytes, bar_b);
            pend_b = true;
        }
        dg_store<P, S, FIN>(sA, tid, kc, v, vn);
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
                    for (int c = 0; c < 2; c++) {
                        const int w = c ? c1 : c0;
                        if (w == 0) continue;
                        // the block's part images: 8 K groups of w rows x 16 bytes each
                        const uint32_t b0 = sB + (uint32_t)(c ? c0 : 0) * KC * 2;
                        const uint32_t lb = (uint32_t)w * 16;
                        const uint32_t dt = tbase + (uint32_t)(c ? c0 : 0);
                        const uint32_t id = idesc_bf16(w);
                        // products A_i M_j, i + j < S, largest first
#pragma unroll
                        for (int o = 0; o < S; o++)
#pragma unroll
                            for (int i = 0; i <= o; i++) {
                                const int j = o - i;
                                const uint64_t ad = smem_desc(sA + i * A_IMG + 2 * ks * A_LBO, A_LBO, 128);
                                const uint64_t bd = smem_desc(b0 + (uint32_t)j * npc * KC * 2 + 2 * ks * lb, lb, 128);
                                mma_bf16(dt, ad, bd, id, (kc > 0 || ks > 0 || o > 0) ? 1u : 0u);
                            }
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
        if (it2 < items) dg_load<P, FIN>(a, it2 / a.npass, kc2, tid, v, vn);
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
            tm_fence_after();
            const int q = warp & 3, h = warp >> 2;
            const int64_t t0 = tile * BM;
            const int ft = (int)(t0 / a.rows);
            const int64_t rt = t0 - (int64_t)ft * a.rows;
            // rows per staging round: the tile's output rows are contiguous in the destination
            // when the tile lies in one array and one pass covers all columns
            // staging: rows of N floats back to back (the block is copied out in order); where N is a
            // multiple of 32 the 8-byte pairs of row r are XOR-swizzled by r % 16, so that the 32
            // rows a warp writes at one column do not all fall in one bank
            const bool swz = (a.N & 31) == 0;
            const int rb = (a.npass == 1 && a.ld == a.N && ft < a.nf && rt + BM <= a.rows)
                               ? (64 * a.N * 4 <= S * A_IMG ? 64 : 32 * a.N * 4 <= S * A_IMG ? 32 : 0) : 0;
            if (rb) {
                // staged epilogue: per round the warps holding rows [rho rb, (rho + 1) rb) move them
                // from TMEM into shared memory (the A images, free now), then all threads copy the
                // rb x N block to its contiguous place in the destination (8-byte stores in order)
                float2* stg2 = reinterpret_cast<float2*>(sm + (sA - smem_addr(sm)));
                float2* dst2 = reinterpret_cast<float2*>(a.dst[ft] + rt * a.ld);
                const int h2 = a.N / 2;
                for (int rho = 0; rho < BM / rb; rho++) {
                    if (q * 32 >= rho * rb && q * 32 < (rho + 1) * rb) {
                        const int rl = q * 32 - rho * rb + lane;          // row within the round
                        const int sw = swz ? (rl & 15) : 0;
                        float2* srow = stg2 + rl * h2;
                        for (int u = h; u < npc / 16; u += 2) {
                            float t[16];
                            tm_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * u), t);
                            tm_wait_ld();
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                const int c = 16 * u + j;          // product columns c, c + 1
                                if (a.fold == 2 && c == 0) {
                                    srow[sw] = make_float2(t[0], 0.f);
                                    srow[(h2 - 1) ^ sw] = make_float2(t[1], 0.f);
                                } else if (c < a.N) {
                                    srow[(c >> 1) ^ sw] = make_float2(t[j], t[j + 1]);
                                }
                            }
                        }
                    }
                    __syncthreads();
                    float2* d2 = dst2 + (int64_t)rho * rb * h2;
                    if (swz) {
                        const int lg = 31 - __clz(h2);                     // h2 is a power of two here
                        for (int e = tid; e < rb * h2; e += NT) {
                            const int r = e >> lg, m = e & (h2 - 1);
                            d2[e] = stg2[(r << lg) + (m ^ (r & 15))];
                        }
                    } else {
                        for (int e = tid; e < rb * h2; e += NT) d2[e] = stg2[e];
                    }
                    __syncthreads();
                }
            } else {
                // direct epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows), column units of 16
                // alternating between the two warp halves, and stores each row's values
                int f = 0;
                int64_t r = 0;
                {
                    const int64_t gr = t0 + 32 * q + lane;
                    f = (int)(gr / a.rows);
                    r = gr - (int64_t)f * a.rows;
                }
                float* out = f < a.nf ? a.dst[f] + r * a.ld : nullptr;
                for (int u = h; u < npc / 16; u += 2) {
                    float t[16];
                    tm_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * u), t);
                    tm_wait_ld();
                    const int n0 = p * pass_cols(S) + 16 * u;
                    if (out) {
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            const int c = n0 + j;          // product columns c, c + 1
                            if (a.fold == 2 && c == 0) {
                                *reinterpret_cast<float2*>(out) = make_float2(t[0], 0.f);
                                *reinterpret_cast<float2*>(out + a.N - 2) = make_float2(t[1], 0.f);
                            } else if (c < a.N) {
                                *reinterpret_cast<float2*>(out + c) = make_float2(t[j], t[j + 1]);
                            }
                        }
                    }
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
    int K = 0, N = 0, nkc = 0, npass = 0, S = 2;
    int Nout = 0, fold = 0;             // output columns written, DgArgs::fold
    int npc[dg::MAXPASS] = {};
    int64_t boff[dg::MAXPASS] = {};
    uint32_t tcols = 0;
    size_t smem = 0;
    int grid = 0;
    void (*kern)(DgArgs) = nullptr;     // k_dft_tc<P, S>, P = pairs per row and warp row
};
struct DftPlan {
    DftOp fwd, inv;
};

template <int S, bool FIN>
static void (*pick_kernel(int K))(DgArgs) {
    return K <= 16 ? k_dft_tc<8, S, FIN> : K <= 32 ? k_dft_tc<16, S, FIN> : k_dft_tc<32, S, FIN>;
}

// M[n][k] (FP64, n < N, k < K) -> images [pass][chunk][part][block][k / 8][n][k % 8] of BF16
static hyb_status make_op(hyb_grid* g, DftOp& op, const std::vector<double>& M, int N, int K, int S, int fold) {
    using namespace dg;
    op.K = K;
    op.N = N;
    op.S = S;
    op.fold = fold;
    op.nkc = (K + KC - 1) / KC;
    const int Np = (N + 15) & ~15, PC = pass_cols(S);
    op.npass = (Np + PC - 1) / PC;
    if (op.npass > MAXPASS) { set_error("DFT-GEMM: n1 too large"); return HYB_EINVAL; }
    size_t total = 0;
    int maxc = 0;
    for (int p = 0; p < op.npass; p++) {
        op.npc[p] = std::min(PC, Np - p * PC);
        op.boff[p] = (int64_t)total;
        total += (size_t)op.nkc * S * op.npc[p] * KC;
        maxc = std::max(maxc, op.npc[p]);
    }
    std::vector<__nv_bfloat16> img(total, __float2bfloat16(0.f));
    for (int p = 0; p < op.npass; p++) {
        const int npc = op.npc[p];
        const int c0 = std::min(256, npc);
        for (int kc = 0; kc < op.nkc; kc++) {
            __nv_bfloat16* base = img.data() + op.boff[p] + (size_t)kc * S * npc * KC;
            for (int nl = 0; nl < npc; nl++) {
                const int blk = nl < c0 ? 0 : 1, w = blk ? npc - c0 : c0, nb = blk ? nl - c0 : nl;
                const size_t boff = (size_t)(blk ? c0 : 0) * KC;
                for (int kl = 0; kl < KC; kl++) {
                    const int n = p * PC + nl, k = kc * KC + kl;
                    float r = (n < N && k < K) ? (float)M[(size_t)n * K + k] : 0.f;
                    const size_t e = boff + ((size_t)(kl >> 3) * w + nb) * 8 + (kl & 7);
                    for (int q = 0; q < S; q++) {        // part q: the rounding of what parts < q leave
                        const __nv_bfloat16 bq = __float2bfloat16(r);
                        r -= __bfloat162float(bq);
                        base[(size_t)q * npc * KC + e] = bq;
                    }
                }
            }
        }
    }
    HYB_CUDA_TRY(cudaMalloc(&op.B, sizeof(__nv_bfloat16) * total));
    HYB_CUDA_TRY(cudaMemcpy(op.B, img.data(), sizeof(__nv_bfloat16) * total, cudaMemcpyHostToDevice));
    op.tcols = maxc <= 256 ? 256 : 512;
    op.smem = 128 + (size_t)off_b(S) + (size_t)maxc * KC * 2 * S;
    op.kern = S == 2 ? (fold == 1 ? pick_kernel<2, true>(K) : pick_kernel<2, false>(K))
                     : (fold == 1 ? pick_kernel<3, true>(K) : pick_kernel<3, false>(K));
    const void* kf = (const void*)op.kern;
    HYB_CUDA_TRY(func_attr_once(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(128 + off_b(S) + PC * KC * 2 * S)));
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
    const int S = g->path == 4 ? 3 : 2;
    // the DC and Nyquist imaginary parts are zero: the forward product's row 1 computes the
    // Nyquist real part (n1 product columns for n1 + 2 outputs), and the inverse reads that part
    // in the DC imaginary slot (K = n1)
    std::vector<double> Ff((size_t)n * n), If((size_t)n * n);
    for (int r = 0; r < n; r++)
        for (int j = 0; j < n; j++) Ff[(size_t)r * n + j] = r == 1 ? F[(size_t)n * n + j] : F[(size_t)r * n + j];
    for (int j = 0; j < n; j++)
        for (int k = 0; k < n; k++) If[(size_t)j * n + k] = k == 1 ? I[(size_t)j * nc + n] : I[(size_t)j * nc + k];
    hyb_status st = make_op(g, P->fwd, Ff, n, n, S, 2);
    P->fwd.Nout = nc;
    if (st == HYB_OK) st = make_op(g, P->inv, If, n, n, S, 1);
    P->inv.Nout = n;
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
    a.N = op.Nout;
    a.ld = ld;
    a.fold = op.fold;
    a.nkc = op.nkc;
    a.npass = op.npass;
    for (int p = 0; p < dg::MAXPASS; p++) { a.npc[p] = op.npc[p]; a.boff[p] = op.boff[p]; }
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
