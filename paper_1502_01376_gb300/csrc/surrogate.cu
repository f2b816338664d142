// surrogate.cu -- a small MLP that learns the NCI growth rate from the root
// solver's data (forward, backward and Adam written here; BF16 weights and
// activations as tensor-core operands, FP32 accumulation, FP32 master
// weights).  Architecture: n_in -> width x depth (tanh) -> 1 (linear).
//
// The GEMMs run on the fifth-generation tensor cores: tcgen05.mma (kind::f16,
// BF16 operands) into FP32 accumulators in tensor memory, 128 x 32 output tiles
// per CTA (narrow, so that the small products still give each SM a dozen warps), operands loaded into the canonical K-major shared-memory layout with
// 16-byte vector loads: every operand is stored with its K index contiguous
// (the epilogues write the activations and dH both batch-major and
// feature-major, and the weights are kept in BF16 both ways).  The network is
// small (widths 16..256), so this is not a roofline-bound path.  The
// elementwise work sits in the GEMM epilogues (bias and tanh; loss, output dH
// and its bias gradient; tanh' and the bias gradient of the layer below), and
// the Adam step sums the gradient parts and writes the BF16 weight copies: a
// training step is 3 launches per layer (forward, dW, dX; no dX below the first
// layer) plus the Adam step.  No sum is taken with atomics: the weight
// gradients (K = batch, split over up to 64 CTAs per tile), the bias gradients
// and the loss are written as per-CTA parts and added in a fixed order, so a
// training run is bit-reproducible.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "hyb_internal.cuh"
#include "tm_dev.cuh"

namespace hyb {
// per-layer offsets and sizes for the gradient sums and the Adam step (passed by value)
constexpr int kMaxLayers = 17;
struct LayerTab {
    int L;
    int nrb;                                          // row blocks of the batch (parts of a bias gradient)
    int64_t w_off[kMaxLayers], wb_off[kMaxLayers];    // parameters; BF16 weight copies
    int64_t ws_w[kMaxLayers], ws_b[kMaxLayers];       // parts of the weight and bias gradients
    int fo[kMaxLayers], fi[kMaxLayers], fop[kMaxLayers], fip[kMaxLayers], split[kMaxLayers];
};
}  // namespace hyb

struct hyb_mlp {
    int n_in = 0, width = 0, depth = 0;   // hidden layers of `width`
    int L = 0;                            // layers = depth + 1
    hyb::LayerTab tab{};
    float* master = nullptr;              // FP32 weights and biases, all layers
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wbf = nullptr;         // BF16 weights [fout_pad][fin_pad] per layer
    __nv_bfloat16* wbt = nullptr;         // BF16 weights transposed [fin_pad][fout_pad] per layer
    float* grad = nullptr;                // FP32 gradients (same layout as master)
    std::vector<size_t> w_off, b_off, wb_off;
    size_t n_params = 0;
    int64_t cap = 0;                      // batch capacity of the activations
    __nv_bfloat16* act = nullptr;         // [L-1][cap][256] BF16 inputs X_l of layers l >= 1
    __nv_bfloat16* actT = nullptr;        // [L-1][256][cap] the same, feature-major
    float* pre = nullptr;                 // [L-1][cap][256] FP32 pre-activations of the hidden layers
    __nv_bfloat16* dhb = nullptr;         // [2][cap][256] BF16 dH (two layers' worth)
    __nv_bfloat16* dhT = nullptr;         // [2][256][cap] the same, feature-major
    float* ws = nullptr;                  // gradient parts: weights (split x fo x fi per layer), biases, loss
    size_t ws_w_size = 0;
    float* loss = nullptr;                // device scalar
    int* err = nullptr;                   // device flag: bit 1 = a bounded wait in a GEMM gave up
    int64_t step = 0;
    int64_t launches = 0;                 // kernels launched so far (hyb_mlp_launch_count)
};

namespace hyb {

// GEMM tiles: 128 x 32 outputs per CTA (tcgen05.mma M = 128, N = 32), K in chunks of 64
constexpr int TM = 128, TN = 32, TKC = 64, GT = 128;
constexpr int LBO_A = TM * 16 + 16, LBO_B = TN * 16 + 16;     // K-group strides (16-byte slots spread)
constexpr int kMaxSplit = 64;

// Epilogues of the GEMM (what happens to an accumulator value v of output (row, col)):
//   EP_PART    part z of a split K: P[z][row][col] = v (row stride N); a CTA with an empty K
//              range writes zeros
//   EP_HIDDEN  h = v + b[col]; pre[row][col] = h; X[row][col] = XT[col][row] = BF16(tanh h)
//              (0 for col >= n)
//   EP_OUTPUT  y = v + b[0] (column 0); out[row] = y; with a target t: d = 2 (y - t) / B,
//              dH[row] = (d, 0, ..., 0) and dHT[0][row] = d in BF16, and per CTA the parts
//              sum (y - t)^2 / B and sum d (loss and bias gradient) at index blockIdx.y
//   EP_DX      dH'[row][col] = dH'T[col][row] = BF16(v (1 - tanh(pre[row][col])^2)) for
//              col < n (else 0), and per CTA the column sums of dH' (bias gradient of the
//              layer below) at [blockIdx.y][col]
enum : int { EP_PART = 0, EP_HIDDEN, EP_OUTPUT, EP_DX };
struct Epi {
    float* c = nullptr;                  // EP_PART output
    const float* bias = nullptr;         // EP_HIDDEN, EP_OUTPUT
    float* pre = nullptr;                // EP_HIDDEN: written; EP_DX: read (pre-activations below)
    __nv_bfloat16* act = nullptr;        // EP_HIDDEN: X (row stride 256); EP_OUTPUT, EP_DX: dH
    __nv_bfloat16* actT = nullptr;       // the same, feature-major (row stride ldT)
    int64_t ldT = 0;
    float* out = nullptr;                // EP_OUTPUT: y (nullable)
    const float* tgt = nullptr;          // EP_OUTPUT: targets (nullable: forward only)
    float* loss_part = nullptr;          // EP_OUTPUT: [row blocks]
    float* db_part = nullptr;            // EP_OUTPUT: [row blocks]; EP_DX: [row blocks][n]
    int n = 0;                           // live columns
    float invB = 0.f;
};

__device__ __forceinline__ uint32_t bf16_bits(float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(x)); }
__device__ __forceinline__ uint32_t bf16_bits(__nv_bfloat16 x) { return (uint32_t)__bfloat16_as_ushort(x); }

// 16-byte slots (row r, group g of 8 k values) of a ROWS x 64 tile: ROWS x 8 slots, ROWS * 8 / GT
// per thread.  All of a thread's global loads are issued before its shared-memory stores, so
// that their latencies overlap (a store between two loads would serialise them).  A source
// whose k index is contiguous is read 16 bytes at a time; the network input (FP32, 6 columns)
// is read element by element and rounded to BF16.
template <int ROWS, typename TA>
__device__ __forceinline__ void gemm_fill(uint32_t dst, int lbo, int rmax, int r0, int k0, int kmax,
                                          const TA* __restrict__ src, int64_t sr, int64_t sk, int tid) {
    constexpr int IT = ROWS * 8 / GT;
    constexpr bool kBF = sizeof(TA) == 2;
    const bool kfast = sk == 1 && (sr & 7) == 0;
    uint4 v[IT];
    uint32_t off[IT];
#pragma unroll
    for (int q = 0; q < IT; q++) {
        const int i = tid + q * GT;
        const int r = kfast ? i >> 3 : i % ROWS, g = kfast ? i & 7 : i / ROWS;
        const int row = r0 + r, k = k0 + 8 * g;
        off[q] = (uint32_t)(g * lbo + 16 * r);
        v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (row < rmax) {
            if (kBF && kfast && k + 8 <= kmax) {
                v[q] = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)row * sr + k));
            } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const uint32_t x = (k + e < kmax) ? bf16_bits(__ldg(src + (int64_t)row * sr + (int64_t)(k + e) * sk)) : 0u;
                    w[e >> 1] |= x << (16 * (e & 1));
                }
                v[q] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < IT; q++)
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                     :: "r"(dst + off[q]), "r"(v[q].x), "r"(v[q].y), "r"(v[q].z), "r"(v[q].w) : "memory");
}

// sum of v over the 32 lanes of a warp (the same butterfly order in every lane)
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// C[m][n] (FP32) = sum_k A(m,k) B(k,n), A(m,k) = a[m*sam + k*sak], B(k,n) = b[k*sbk + n*sbn]
// (BF16, or FP32 rounded to BF16 on the way in: the network input), K a multiple of 16,
// entries with k >= kmax read as zero.  Split K (EP_PART only): block z handles k in
// [z*kchunk, (z+1)*kchunk).
// Per 64-wide K chunk the 128 threads load the A and B tiles into shared memory in the
// canonical K-major layout without swizzle (8 x 16-byte core matrices; 16-byte slots (row, k/8)),
// one thread issues the k-steps of tcgen05.mma into the 128 x 32 FP32 accumulator in TMEM and
// commits them to an mbarrier, and after the last chunk each warp reads its 32 rows with
// tcgen05.ld into the epilogue.  Waits are bounded: on time-out bit 1 of *err is set and the
// CTA skips the rest, drains and frees its TMEM.
template <int EP, typename TA, typename TB>
__global__ void __launch_bounds__(GT) k_gemm_tc(int M, int N, int K, int kmax, const TA* __restrict__ a, int64_t sam, int64_t sak,
                                                const TB* __restrict__ b, int64_t sbk, int64_t sbn, Epi ep, int kchunk, int* err) {
    __shared__ __align__(128) unsigned char sbuf[8 * LBO_A + 8 * LBO_B];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    __shared__ float s_red[4][TN];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sA = smem_addr(sbuf), sB = sA + 8 * LBO_A, mb = smem_addr(&bar);
    if (warp == 0) {
        tm_alloc(smem_addr(&s_taddr), TN);
        tm_relinquish();
    }
    if (tid == 0) {
        mbar_init(mb, 1);
        mbar_fence_init();
        s_abort = 0;
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tbase = s_taddr;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    uint32_t ph = 0;
    bool pend = false, abort = false, any = false;
    for (int k0 = kb; k0 < ke && !abort; k0 += TKC) {
        gemm_fill<TM, TA>(sA, LBO_A, M, m0, k0, kmax, a, sam, sak, tid);
        gemm_fill<TN, TB>(sB, LBO_B, N, n0, k0, kmax, b, sbn, sbk, tid);
        fence_proxy_async_smem();
        tm_fence_before();
        __syncthreads();
        if (tid == 0) {
            tm_fence_after();
            const int nks = min(TKC, ke - k0) / 16;
            for (int ks = 0; ks < nks; ks++)
                mma_bf16(tbase, smem_desc(sA + 2 * ks * LBO_A, LBO_A, 128), smem_desc(sB + 2 * ks * LBO_B, LBO_B, 128),
                         idesc_bf16(TN), (k0 > kb || ks > 0) ? 1u : 0u);
            mma_commit(mb);
            pend = true;
            mbar_wait(mb, ph, err, &s_abort);
            if (!s_abort) {
                ph ^= 1;
                pend = false;
            }
        }
        __syncthreads();
        abort = s_abort != 0;
        any = true;
    }
    if (!abort) {
        if (any) tm_fence_after();
        const int row = m0 + 32 * warp + lane;
        const bool live = row < M;
        const int nchunk = EP == EP_OUTPUT ? 1 : TN / 16;
        for (int u = 0; u < nchunk; u++) {
            float t[16];
            if (any) {
                tm_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * u), t);
                tm_wait_ld();
            } else {
#pragma unroll
                for (int j = 0; j < 16; j++) t[j] = 0.f;
            }
            const int c0 = n0 + 16 * u;
            if (EP == EP_PART) {
                if (live && c0 < N) {
                    float* p = ep.c + (int64_t)blockIdx.z * M * N + (int64_t)row * N + c0;
                    if ((N & 3) == 0 && c0 + 16 <= N) {
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            reinterpret_cast<float4*>(p)[j] = make_float4(t[4 * j], t[4 * j + 1], t[4 * j + 2], t[4 * j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            if (c0 + j < N) p[j] = t[j];
                    }
                }
            } else if (EP == EP_HIDDEN) {
                if (live && c0 < N) {
                    float h[16];
                    uint32_t q[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const int col = c0 + j;
                        h[j] = t[j] + (col < ep.n ? __ldg(ep.bias + col) : 0.f);
                        q[j >> 1] |= (col < ep.n ? bf16_bits(tanhf(h[j])) : 0u) << (16 * (j & 1));
                    }
                    float4* pp = reinterpret_cast<float4*>(ep.pre + (int64_t)row * 256 + c0);
#pragma unroll
                    for (int j = 0; j < 4; j++) pp[j] = make_float4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
                    uint4* pa = reinterpret_cast<uint4*>(ep.act + (int64_t)row * 256 + c0);
                    pa[0] = make_uint4(q[0], q[1], q[2], q[3]);
                    pa[1] = make_uint4(q[4], q[5], q[6], q[7]);
                    unsigned short* pt = reinterpret_cast<unsigned short*>(ep.actT) + (int64_t)c0 * ep.ldT + row;
#pragma unroll
                    for (int j = 0; j < 16; j++) pt[(int64_t)j * ep.ldT] = (unsigned short)(q[j >> 1] >> (16 * (j & 1)));
                }
            } else if (EP == EP_OUTPUT) {
                const float y = t[0] + __ldg(ep.bias);
                if (live && ep.out) ep.out[row] = y;
                if (ep.tgt) {
                    const float dd = live ? y - ep.tgt[row] : 0.f;
                    const float d = 2.f * dd * ep.invB;
                    if (live) {
                        const uint32_t db = bf16_bits(d);
                        uint4* pa = reinterpret_cast<uint4*>(ep.act + (int64_t)row * 256);
                        pa[0] = make_uint4(db, 0u, 0u, 0u);
                        pa[1] = make_uint4(0u, 0u, 0u, 0u);
                        reinterpret_cast<unsigned short*>(ep.actT)[row] = (unsigned short)db;
                    }
                    const float l = warp_sum(dd * dd * ep.invB), sd = warp_sum(d);
                    if (lane == 0) { s_red[warp][0] = l; s_red[warp][1] = sd; }
                    __syncthreads();
                    if (tid == 0) {
                        ep.loss_part[blockIdx.y] = (s_red[0][0] + s_red[1][0]) + (s_red[2][0] + s_red[3][0]);
                        ep.db_part[blockIdx.y] = (s_red[0][1] + s_red[1][1]) + (s_red[2][1] + s_red[3][1]);
                    }
                }
            } else {   // EP_DX
                if (c0 < N) {
                    float d[16];
                    uint32_t q[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                    if (live) {
                        const float4* pp = reinterpret_cast<const float4*>(ep.pre + (int64_t)row * 256 + c0);
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const float4 h = pp[j];
                            const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const float th = tanhf(hv[i]);
                                d[4 * j + i] = (c0 + 4 * j + i < ep.n) ? t[4 * j + i] * (1.f - th * th) : 0.f;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 16; j++) q[j >> 1] |= bf16_bits(d[j]) << (16 * (j & 1));
                        uint4* pa = reinterpret_cast<uint4*>(ep.act + (int64_t)row * 256 + c0);
                        pa[0] = make_uint4(q[0], q[1], q[2], q[3]);
                        pa[1] = make_uint4(q[4], q[5], q[6], q[7]);
                        unsigned short* pt = reinterpret_cast<unsigned short*>(ep.actT) + (int64_t)c0 * ep.ldT + row;
#pragma unroll
                        for (int j = 0; j < 16; j++) pt[(int64_t)j * ep.ldT] = (unsigned short)(q[j >> 1] >> (16 * (j & 1)));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j++) d[j] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const float sj = warp_sum(d[j]);
                        if (lane == 0) s_red[warp][16 * u + j] = sj;
                    }
                }
            }
        }
        if (EP == EP_DX) {
            __syncthreads();
            if (tid < TN && n0 + tid < ep.n)
                ep.db_part[(int64_t)blockIdx.y * ep.n + n0 + tid] = (s_red[0][tid] + s_red[1][tid]) + (s_red[2][tid] + s_red[3][tid]);
        }
    }
    if (tid == 0 && pend) mbar_drain(mb, ph);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, TN);
}

// K is rounded up to 16 (the MMA depth); entries with k >= K read as zero.
static int split_of(int M, int N, int K) {
    const int Kp = (K + 15) & ~15;
    const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
    int split = 1;
    while (split < kMaxSplit && tiles * split < 600 && Kp / (split * 2) >= 256) split *= 2;
    return split;
}
// Few output tiles and a long K (the weight gradients: K = batch) are split along K into
// parts that the caller adds up (EP_PART).
template <int EP, typename TA, typename TB>
static void gemm(int M, int N, int K, const TA* a, int64_t sam, int64_t sak, const TB* b, int64_t sbk, int64_t sbn,
                 const Epi& ep, cudaStream_t s, int64_t& launches, int* err) {
    const int Kp = (K + 15) & ~15;
    const int split = EP == EP_PART ? split_of(M, N, K) : 1;
    const int kchunk = (((Kp + split - 1) / split + 15) & ~15);     // the parts cover all of K
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, split);
    k_gemm_tc<EP, TA, TB><<<grid, GT, 0, s>>>(M, N, Kp, K, a, sam, sak, b, sbk, sbn, ep, kchunk, err);
    launches++;
}

// Gradient sums in a fixed order (the split-K parts of a weight gradient, the row-block parts of
// a bias gradient, the loss parts); with update != 0 also the Adam step on every parameter and
// the BF16 copies of the updated weights (zero-padded, both layouts; the padding was written by
// refresh()).  Without it the sums go to g (the gradients of hyb_mlp_gradients).
__global__ void k_grad_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ ws, const float* __restrict__ loss_part, float* __restrict__ loss,
                            int64_t n, int update, float lr, float b1, float b2, float eps, float c1, float c2, LayerTab tab,
                            __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) {
        float s = 0.f;
        for (int y = 0; y < tab.nrb; y++) s += loss_part[y];
        *loss = s;
    }
    if (i >= n) return;
    int l = 0;
    while (l + 1 < tab.L && i >= tab.w_off[l + 1]) l++;
    const int64_t loc = i - tab.w_off[l];
    const int64_t nw = (int64_t)tab.fo[l] * tab.fi[l];
    float gi = 0.f;
    if (loc < nw) {
        const float* p = ws + tab.ws_w[l] + loc;
        for (int z = 0; z < tab.split[l]; z++) gi += p[z * nw];
    } else {
        const float* p = ws + tab.ws_b[l] + (loc - nw);
        for (int y = 0; y < tab.nrb; y++) gi += p[(int64_t)y * tab.fo[l]];
    }
    if (!update) {
        g[i] = gi;
        return;
    }
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (loc < nw) {
        const int r = (int)(loc / tab.fi[l]), c = (int)(loc % tab.fi[l]);
        const __nv_bfloat16 q = __float2bfloat16(wi);
        wb[tab.wb_off[l] + (int64_t)r * tab.fip[l] + c] = q;
        wt[tab.wb_off[l] + (int64_t)c * tab.fop[l] + r] = q;
    }
}

// BF16 copies of the weights, zero-padded to [fout_pad][fin_pad] and [fin_pad][fout_pad]
// (at creation and on new parameters)
__global__ void k_refresh(const float* __restrict__ w, int fout, int fin, int fout_p, int fin_p, __nv_bfloat16* __restrict__ wb,
                          __nv_bfloat16* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= fout_p * fin_p) return;
    const int r = i / fin_p, c = i % fin_p;
    const __nv_bfloat16 q = __float2bfloat16((r < fout && c < fin) ? w[r * fin + c] : 0.f);
    wb[i] = q;
    wt[c * fout_p + r] = q;
}

static int pad16(int v) { return (v + 15) & ~15; }

static int layer_in(const hyb_mlp* m, int l) { return l == 0 ? m->n_in : m->width; }
static int layer_out(const hyb_mlp* m, int l) { return l == m->L - 1 ? 1 : m->width; }

static hyb_status refresh(hyb_mlp* m, cudaStream_t s) {
    for (int l = 0; l < m->L; l++) {
        const int fo = layer_out(m, l), fi = layer_in(m, l), fop = pad16(fo), fip = pad16(fi);
        k_refresh<<<(fop * fip + 255) / 256, 256, 0, s>>>(m->master + m->w_off[l], fo, fi, fop, fip, m->wbf + m->wb_off[l],
                                                          m->wbt + m->wb_off[l]);
        m->launches++;
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

static hyb_status ensure_cap(hyb_mlp* m, int64_t B) {
    if (B <= m->cap) return HYB_OK;
    if (m->act) { cudaFree(m->act); cudaFree(m->actT); cudaFree(m->pre); cudaFree(m->dhb); cudaFree(m->dhT); cudaFree(m->ws); }
    m->act = m->actT = m->dhb = m->dhT = nullptr;
    m->pre = m->ws = nullptr;
    m->cap = 0;
    const int64_t cap = ((B + 127) / 128) * 128;
    const size_t na = (size_t)std::max(1, m->L - 1) * cap * 256;
    const size_t nrb = (size_t)(cap / 128);
    size_t nb = 0;
    for (int l = 0; l < m->L; l++) nb += nrb * layer_out(m, l);
    HYB_CUDA_TRY(cudaMalloc(&m->act, sizeof(__nv_bfloat16) * na));
    HYB_CUDA_TRY(cudaMalloc(&m->actT, sizeof(__nv_bfloat16) * na));
    HYB_CUDA_TRY(cudaMalloc(&m->pre, sizeof(float) * na));
    HYB_CUDA_TRY(cudaMalloc(&m->dhb, sizeof(__nv_bfloat16) * 2 * (size_t)cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->dhT, sizeof(__nv_bfloat16) * 2 * (size_t)cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->ws, sizeof(float) * (m->ws_w_size + nb + nrb)));
    // bias parts start after the weight parts, the loss parts after the bias parts
    size_t off = m->ws_w_size;
    for (int l = 0; l < m->L; l++) { m->tab.ws_b[l] = (int64_t)off; off += nrb * layer_out(m, l); }
    m->cap = cap;
    return HYB_OK;
}

static float* loss_parts(const hyb_mlp* m) { return m->ws + m->tab.ws_b[m->L - 1] + (size_t)(m->cap / 128) * layer_out(m, m->L - 1); }

// input of layer l >= 1 (BF16 activations of layer l - 1): row-major [cap][256] and feature-major [256][cap]
static __nv_bfloat16* act_in(const hyb_mlp* m, int l) { return m->act + (size_t)(l - 1) * m->cap * 256; }
static __nv_bfloat16* actT_in(const hyb_mlp* m, int l) { return m->actT + (size_t)(l - 1) * m->cap * 256; }
// dH of layer l (BF16): two buffers of each layout, so that the dX product of layer l reads one
// while its epilogue writes dH of layer l - 1 into the other
static int dh_buf(const hyb_mlp* m, int l) { return (m->L - 1 - l) & 1; }
static __nv_bfloat16* dh_of(const hyb_mlp* m, int l) { return m->dhb + (size_t)dh_buf(m, l) * m->cap * 256; }
static __nv_bfloat16* dhT_of(const hyb_mlp* m, int l) { return m->dhT + (size_t)dh_buf(m, l) * m->cap * 256; }

// forward pass: one GEMM per layer, bias and tanh in its epilogue; with a target the output
// layer's epilogue also forms dH of the output layer and the parts of the loss and its bias gradient
static hyb_status forward(hyb_mlp* m, const float* x, int64_t B, float* y, const float* tgt, cudaStream_t s) {
    hyb_status st = ensure_cap(m, B);
    if (st != HYB_OK) return st;
    const int64_t cap = m->cap;
    for (int l = 0; l < m->L; l++) {
        const int fi = pad16(layer_in(m, l)), fo = pad16(layer_out(m, l));
        const __nv_bfloat16* W = m->wbf + m->wb_off[l];
        Epi ep;
        ep.bias = m->master + m->b_off[l];
        ep.n = layer_out(m, l);
        ep.invB = 1.f / (float)B;
        ep.ldT = cap;
        // H[B][fo] = X[B][fi] W^T, W stored [fo][fi]
        if (l < m->L - 1) {
            ep.pre = m->pre + (size_t)l * cap * 256;
            ep.act = act_in(m, l + 1);
            ep.actT = actT_in(m, l + 1);
            if (l == 0) gemm<EP_HIDDEN>((int)B, fo, fi, x, m->n_in, 1, W, 1, fi, ep, s, m->launches, m->err);
            else gemm<EP_HIDDEN>((int)B, fo, fi, act_in(m, l), 256, 1, W, 1, fi, ep, s, m->launches, m->err);
        } else {
            ep.out = y;
            ep.tgt = tgt;
            ep.loss_part = loss_parts(m);
            ep.db_part = m->ws + m->tab.ws_b[l];
            ep.act = dh_of(m, l);
            ep.actT = dhT_of(m, l);
            if (l == 0) gemm<EP_OUTPUT>((int)B, fo, fi, x, m->n_in, 1, W, 1, fi, ep, s, m->launches, m->err);
            else gemm<EP_OUTPUT>((int)B, fo, fi, act_in(m, l), 256, 1, W, 1, fi, ep, s, m->launches, m->err);
        }
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

// backward pass after forward(.., tgt): per layer the parts of the weight gradient dW = dH^T X
// (split K) and, below the first layer, dX = dH W with tanh' and the parts of the bias
// gradient of the layer below in the epilogue
static hyb_status backward(hyb_mlp* m, const float* x, int64_t B, cudaStream_t s) {
    const int64_t cap = m->cap;
    m->tab.nrb = (int)((B + TM - 1) / TM);
    for (int l = m->L - 1; l >= 0; l--) {
        const int fi = pad16(layer_in(m, l)), fo = pad16(layer_out(m, l));
        const int ni = layer_in(m, l), no = layer_out(m, l);
        Epi ep;
        ep.c = m->ws + m->tab.ws_w[l];
        m->tab.split[l] = split_of(no, ni, (int)B);
        // dW[no][ni] = dH^T X: M = no, N = ni, K = B, both operands read batch-contiguous
        if (l == 0) gemm<EP_PART>(no, ni, (int)B, dhT_of(m, l), cap, 1, x, m->n_in, 1, ep, s, m->launches, m->err);
        else gemm<EP_PART>(no, ni, (int)B, dhT_of(m, l), cap, 1, actT_in(m, l), 1, cap, ep, s, m->launches, m->err);
        if (l > 0) {
            // dX[B][fi] = dH[B][fo] W[fo][fi] (W read transposed, K = fo contiguous), then dH of layer l - 1
            Epi ed;
            ed.pre = m->pre + (size_t)(l - 1) * cap * 256;
            ed.act = dh_of(m, l - 1);
            ed.actT = dhT_of(m, l - 1);
            ed.ldT = cap;
            ed.db_part = m->ws + m->tab.ws_b[l - 1];
            ed.n = ni;
            gemm<EP_DX>((int)B, fi, fo, dh_of(m, l), 256, 1, m->wbt + m->wb_off[l], 1, fo, ed, s, m->launches, m->err);
        }
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

// the gradient sums (and with update the Adam step) over all parameters: one launch
static hyb_status reduce_update(hyb_mlp* m, int update, float lr, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    if (update) {
        m->step++;
        c1 = 1.f - powf(b1, (float)m->step);
        c2 = 1.f - powf(b2, (float)m->step);
    }
    k_grad_adam<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->master, m->grad, m->adam_m, m->adam_v, m->ws, loss_parts(m),
                                                                     m->loss, (int64_t)m->n_params, update, lr, b1, b2, 1e-8f, c1,
                                                                     c2, m->tab, m->wbf, m->wbt);
    m->launches++;
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" {

hyb_status hyb_mlp_create(int n_in, int width, int depth, const float* init_params, hyb_mlp** out) {
    if (!out || n_in < 1 || n_in > 256 || width < 1 || width > 256 || depth < 1 || depth > kMaxLayers - 1) {
        set_error("hyb_mlp_create: bad sizes");
        return HYB_EINVAL;
    }
    *out = nullptr;
    hyb_mlp* m = new hyb_mlp();
    m->n_in = n_in; m->width = width; m->depth = depth; m->L = depth + 1;
    size_t off = 0, woff = 0, wsw = 0;
    m->tab.L = m->L;
    for (int l = 0; l < m->L; l++) {
        const int fi = layer_in(m, l), fo = layer_out(m, l);
        m->w_off.push_back(off); off += (size_t)fo * fi;
        m->b_off.push_back(off); off += fo;
        m->wb_off.push_back(woff); woff += (size_t)pad16(fo) * pad16(fi);
        m->tab.w_off[l] = (int64_t)m->w_off[l];
        m->tab.wb_off[l] = (int64_t)m->wb_off[l];
        m->tab.ws_w[l] = (int64_t)wsw; wsw += (size_t)kMaxSplit * fo * fi;
        m->tab.fo[l] = fo;
        m->tab.fi[l] = fi;
        m->tab.fop[l] = pad16(fo);
        m->tab.fip[l] = pad16(fi);
    }
    m->n_params = off;
    m->ws_w_size = wsw;
    cudaError_t e = cudaMalloc(&m->master, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->wbf, sizeof(__nv_bfloat16) * woff);
    if (e == cudaSuccess) e = cudaMalloc(&m->wbt, sizeof(__nv_bfloat16) * woff);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * off);
    if (e == cudaSuccess && init_params) e = cudaMemcpy(m->master, init_params, sizeof(float) * off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { hyb_status st = cuda_fail(e, "hyb_mlp_create"); hyb_mlp_destroy(m); return st; }
    if (!init_params) cudaMemset(m->master, 0, sizeof(float) * off);
    hyb_status st = refresh(m, nullptr);
    if (st != HYB_OK) { hyb_mlp_destroy(m); return st; }
    cudaDeviceSynchronize();
    *out = m;
    return HYB_OK;
}

int64_t hyb_mlp_num_params(const hyb_mlp* m) { return m ? (int64_t)m->n_params : 0; }

hyb_status hyb_mlp_set_params(hyb_mlp* m, const float* params_host) {
    if (!m || !params_host) { set_error("null argument"); return HYB_EINVAL; }
    HYB_CUDA_TRY(cudaMemcpy(m->master, params_host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
    return refresh(m, nullptr);
}

hyb_status hyb_mlp_get_params(hyb_mlp* m, float* params_host) {
    if (!m || !params_host) { set_error("null argument"); return HYB_EINVAL; }
    HYB_CUDA_TRY(cudaDeviceSynchronize());
    HYB_CUDA_TRY(cudaMemcpy(params_host, m->master, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    int h = 0;
    HYB_CUDA_TRY(cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(m->err, 0, sizeof(int));
        set_error("a bounded device-side wait in the surrogate's GEMMs gave up");
        return HYB_ETIMEOUT;
    }
    return HYB_OK;
}

hyb_status hyb_mlp_forward(hyb_mlp* m, const float* x, int64_t B, float* y, void* stream) {
    if (!m || !x || !y || B < 1) { set_error("hyb_mlp_forward: bad arguments"); return HYB_EINVAL; }
    return forward(m, x, B, y, nullptr, (cudaStream_t)stream);
}

hyb_status hyb_mlp_gradients(hyb_mlp* m, const float* x, const float* target, int64_t B, float* grad_host, float* loss_host,
                             void* stream) {
    if (!m || !x || !target || B < 1) { set_error("hyb_mlp_gradients: bad arguments"); return HYB_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    hyb_status st = forward(m, x, B, nullptr, target, s);
    if (st == HYB_OK) st = backward(m, x, B, s);
    if (st == HYB_OK) st = reduce_update(m, 0, 0.f, s);
    if (st != HYB_OK) return st;
    HYB_CUDA_TRY(cudaStreamSynchronize(s));
    if (grad_host) HYB_CUDA_TRY(cudaMemcpy(grad_host, m->grad, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    if (loss_host) HYB_CUDA_TRY(cudaMemcpy(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return HYB_OK;
}

hyb_status hyb_mlp_train_step(hyb_mlp* m, const float* x, const float* target, int64_t B, float lr, float* loss_dev,
                              void* stream) {
    if (!m || !x || !target || B < 1) { set_error("hyb_mlp_train_step: bad arguments"); return HYB_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    hyb_status st = forward(m, x, B, nullptr, target, s);
    if (st == HYB_OK) st = backward(m, x, B, s);
    if (st == HYB_OK) st = reduce_update(m, 1, lr, s);
    if (st != HYB_OK) return st;
    if (loss_dev) HYB_CUDA_TRY(cudaMemcpyAsync(loss_dev, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return HYB_OK;
}

int64_t hyb_mlp_launch_count(const hyb_mlp* m) { return m ? m->launches : 0; }

hyb_status hyb_mlp_destroy(hyb_mlp* m) {
    if (!m) return HYB_OK;
    cudaDeviceSynchronize();
    cudaFree(m->master); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->grad); cudaFree(m->wbf); cudaFree(m->wbt);
    cudaFree(m->loss);
    cudaFree(m->err);
    if (m->act) { cudaFree(m->act); cudaFree(m->actT); cudaFree(m->pre); cudaFree(m->dhb); cudaFree(m->dhT); cudaFree(m->ws); }
    delete m;
    return HYB_OK;
}

}  // extern "C"
