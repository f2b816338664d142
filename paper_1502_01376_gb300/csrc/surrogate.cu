// surrogate.cu -- a small MLP that learns the NCI growth rate from the root
// solver's data (forward, backward and Adam written here; BF16 weights and
// activations as tensor-core operands, FP32 accumulation, FP32 master
// weights).  Architecture: n_in -> width x depth (tanh) -> 1 (linear).
//
// The GEMMs run on the fifth-generation tensor cores: tcgen05.mma (kind::f16,
// BF16 operands) into FP32 accumulators in tensor memory, 128 x 64 output tiles
// per CTA, operands gathered into shared memory from any strides (the weight
// gradients read the activations transposed); the network is small (widths
// 16..256), so this is not a roofline-bound path.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "hyb_internal.cuh"
#include "tm_dev.cuh"

struct hyb_mlp {
    int n_in = 0, width = 0, depth = 0;   // hidden layers of `width`
    int kin = 0;                          // n_in padded to 16
    int L = 0;                            // layers = depth + 1
    std::vector<int> fin, fout;           // per layer, padded to 16
    float* master = nullptr;              // FP32 weights and biases, all layers
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wbf = nullptr;         // BF16 copies of the weights
    float* grad = nullptr;                // FP32 gradients (same layout as master)
    std::vector<size_t> w_off, b_off, wb_off;
    size_t n_params = 0;
    int64_t cap = 0;                      // batch capacity of the activations
    __nv_bfloat16* act = nullptr;         // [L+1][cap][256] BF16 layer inputs (X_l)
    float* pre = nullptr;                 // [L][cap][256] FP32 pre-activations
    float* dh = nullptr;                  // [cap][256] FP32 dH of the current layer
    __nv_bfloat16* dhb = nullptr;         // BF16 copy of dH
    float* dx = nullptr;                  // [cap][256] FP32 dX
    float* loss = nullptr;                // device scalar
    int* err = nullptr;                   // device flag: bit 1 = a bounded wait in a GEMM gave up
    int64_t step = 0;
    int64_t launches = 0;                 // kernels launched so far (hyb_mlp_launch_count)
};

namespace hyb {

// GEMM tiles: 128 x 64 outputs per CTA (tcgen05.mma M = 128, N = 64), K in chunks of 64
constexpr int TM = 128, TN = 64, TKC = 64, GT = 128;
constexpr int LBO_A = TM * 16 + 16, LBO_B = TN * 16 + 16;     // K-group strides (16-byte slots spread)

// C[m][n] (FP32) = sum_k A(m,k) B(k,n), A(m,k) = a[m*sam + k*sak], B(k,n) = b[k*sbk + n*sbn]
// (BF16), K a multiple of 16, entries with k >= kmax read as zero; accumulate into C if
// acc != 0.  Split K: block z handles k in [z*kchunk, (z+1)*kchunk) and, when gridDim.z > 1,
// adds its partial sums atomically (C then holds the caller's zero or previous values).
// Per 64-wide K chunk the 128 threads gather the A and B tiles into shared memory in the
// canonical K-major layout without swizzle (8 x 16-byte core matrices; 16-byte slots (row, k/8),
// filled along whichever index of the source is contiguous), one thread issues the k-steps of
// tcgen05.mma into the 128 x 64 FP32 accumulator in TMEM and commits them to an mbarrier, and
// after the last chunk each warp reads its 32 rows with tcgen05.ld.  Waits are bounded: on
// time-out bit 1 of *err is set and the CTA skips the rest, drains and frees its TMEM.
__device__ __forceinline__ void gemm_fill(uint32_t dst, int lbo, int rows, int rmax, int r0, int k0, int kmax,
                                          const __nv_bfloat16* __restrict__ src, int64_t sr, int64_t sk, int tid) {
    // 16-byte slots (row r, group g of 8 k values): rows x 8 slots
    const bool kfast = sk == 1 && (sr & 7) == 0;
    for (int i = tid; i < rows * 8; i += GT) {
        const int r = kfast ? i >> 3 : i % rows, g = kfast ? i & 7 : i / rows;
        const int row = r0 + r, k = k0 + 8 * g;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < rmax) {
            if (kfast && k + 8 <= kmax) {
                v = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)row * sr + k));
            } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const uint32_t x = (k + e < kmax) ? (uint32_t)__bfloat16_as_ushort(src[(int64_t)row * sr + (int64_t)(k + e) * sk]) : 0u;
                    w[e >> 1] |= x << (16 * (e & 1));
                }
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                     :: "r"(dst + (uint32_t)(g * lbo + 16 * r)), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
    }
}

__global__ void __launch_bounds__(GT) k_gemm_tc(int M, int N, int K, int kmax, const __nv_bfloat16* __restrict__ a, int64_t sam, int64_t sak,
                                                const __nv_bfloat16* __restrict__ b, int64_t sbk, int64_t sbn,
                                                float* __restrict__ c, int64_t scm, int acc, int kchunk, int* err) {
    __shared__ __align__(128) unsigned char sbuf[8 * LBO_A + 8 * LBO_B];
    __shared__ uint64_t bar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
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
        gemm_fill(sA, LBO_A, TM, M, m0, k0, kmax, a, sam, sak, tid);
        gemm_fill(sB, LBO_B, TN, N, n0, k0, kmax, b, sbn, sbk, tid);
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
    if (any && !abort) {
        tm_fence_after();
        const int row = m0 + 32 * warp + lane;
#pragma unroll
        for (int u = 0; u < TN / 16; u++) {
            float t[16];
            tm_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * u), t);
            tm_wait_ld();
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int col = n0 + 16 * u + j;
                    if (col < N) {
                        float* p = c + (int64_t)row * scm + col;
                        if (gridDim.z > 1) atomicAdd(p, t[j]);
                        else *p = acc ? *p + t[j] : t[j];
                    }
                }
            }
        }
    }
    if (tid == 0 && pend) mbar_drain(mb, ph);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tbase, TN);
}

// K is rounded up to 16 (the MMA depth); entries with k >= K read as zero
// Few output tiles and a long K (the weight gradients: K = batch) are split along K
// over up to 64 blocks per tile, the partial sums added atomically into C.
static void gemm(int M, int N, int K, const __nv_bfloat16* a, int64_t sam, int64_t sak, const __nv_bfloat16* b, int64_t sbk,
                 int64_t sbn, float* c, int64_t scm, int acc, cudaStream_t s, int64_t& launches, int* err) {
    const int Kp = (K + 15) & ~15;
    const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
    int split = 1;
    while (split < 64 && tiles * split < 600 && Kp / (split * 2) >= 256) split *= 2;
    const int kchunk = ((Kp / split + 15) & ~15);
    if (split > 1 && !acc) cudaMemsetAsync(c, 0, sizeof(float) * (size_t)M * scm, s);   // rows of stride scm >= N
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, split);
    k_gemm_tc<<<grid, GT, 0, s>>>(M, N, Kp, K, a, sam, sak, b, sbk, sbn, c, scm, acc, kchunk, err);
    launches++;
}

// x (FP32 [B][n_in]) -> BF16 [B][kin] with zero padding
__global__ void k_pack_input(const float* __restrict__ x, int64_t B, int n_in, int kin, __nv_bfloat16* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * kin) return;
    const int64_t r = i / kin;
    const int c = (int)(i % kin);
    out[r * 256 + c] = __float2bfloat16(c < n_in ? x[r * n_in + c] : 0.f);
}

// pre += bias; act = tanh(pre) (BF16) for hidden layers
__global__ void k_bias_act(float* __restrict__ pre, const float* __restrict__ bias, int64_t B, int n, int fout, int hidden,
                           __nv_bfloat16* __restrict__ act, float* __restrict__ yout) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * fout) return;
    const int64_t r = i / fout;
    const int c = (int)(i % fout);
    float v = pre[r * 256 + c] + (c < n ? bias[c] : 0.f);
    pre[r * 256 + c] = v;
    if (hidden) act[r * 256 + c] = __float2bfloat16(c < n ? tanhf(v) : 0.f);
    else if (c == 0 && yout) yout[r] = v;
}

// output layer: dH = 2 (y - t) / B, loss += (y - t)^2 / B
__global__ void k_loss(const float* __restrict__ pre, const float* __restrict__ tgt, int64_t B, float* __restrict__ dh,
                       float* __restrict__ loss) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.f;
    if (r < B) {
        const float d = pre[r * 256] - tgt[r];
        for (int c = 0; c < 16; c++) dh[r * 256 + c] = (c == 0) ? 2.f * d / (float)B : 0.f;
        l = d * d / (float)B;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dH_{l-1} = dX_l * (1 - tanh(pre)^2), only the first n columns are live
__global__ void k_act_back(const float* __restrict__ dx, const float* __restrict__ pre, int64_t B, int n, int fout,
                           float* __restrict__ dh) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * fout) return;
    const int64_t r = i / fout;
    const int c = (int)(i % fout);
    const float th = tanhf(pre[r * 256 + c]);
    dh[r * 256 + c] = (c < n) ? dx[r * 256 + c] * (1.f - th * th) : 0.f;
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// db[c] = sum_r dh[r][c]
__global__ void k_colsum(const float* __restrict__ dh, int64_t B, int n, float* __restrict__ db) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) s += dh[r * 256 + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
        if (c < n) db[c] = t;
    }
}

// copy a [fout][fin] FP32 gradient block out of a [fout_pad][256]-strided product
__global__ void k_copy_grad(const float* __restrict__ src, int rows, int cols, int64_t sstride, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    dst[i] = src[(int64_t)(i / cols) * sstride + i % cols];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of the weights, zero-padded to [fout_pad][fin_pad]
__global__ void k_refresh(const float* __restrict__ w, int fout, int fin, int fout_p, int fin_p, __nv_bfloat16* __restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= fout_p * fin_p) return;
    const int r = i / fin_p, c = i % fin_p;
    wb[i] = __float2bfloat16((r < fout && c < fin) ? w[r * fin + c] : 0.f);
}

static int pad16(int v) { return (v + 15) & ~15; }

static int layer_in(const hyb_mlp* m, int l) { return l == 0 ? m->n_in : m->width; }
static int layer_out(const hyb_mlp* m, int l) { return l == m->L - 1 ? 1 : m->width; }

static hyb_status refresh(hyb_mlp* m, cudaStream_t s) {
    for (int l = 0; l < m->L; l++) {
        const int fo = layer_out(m, l), fi = layer_in(m, l), fop = pad16(fo), fip = pad16(fi);
        k_refresh<<<(fop * fip + 255) / 256, 256, 0, s>>>(m->master + m->w_off[l], fo, fi, fop, fip, m->wbf + m->wb_off[l]);
        m->launches++;
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

static hyb_status ensure_cap(hyb_mlp* m, int64_t B) {
    if (B <= m->cap) return HYB_OK;
    if (m->act) { cudaFree(m->act); cudaFree(m->pre); cudaFree(m->dh); cudaFree(m->dhb); cudaFree(m->dx); }
    m->act = nullptr;
    // at least 256 rows: dx also holds the weight gradient of a layer (up to 256 x 256)
    const int64_t cap = std::max<int64_t>(256, ((B + 63) / 64) * 64);
    HYB_CUDA_TRY(cudaMalloc(&m->act, sizeof(__nv_bfloat16) * (size_t)(m->L + 1) * cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->pre, sizeof(float) * (size_t)m->L * cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->dh, sizeof(float) * (size_t)cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->dhb, sizeof(__nv_bfloat16) * (size_t)cap * 256));
    HYB_CUDA_TRY(cudaMalloc(&m->dx, sizeof(float) * (size_t)cap * 256));
    HYB_CUDA_TRY(cudaMemset(m->act, 0, sizeof(__nv_bfloat16) * (size_t)(m->L + 1) * cap * 256));
    m->cap = cap;
    return HYB_OK;
}

static hyb_status forward(hyb_mlp* m, const float* x, int64_t B, float* y, cudaStream_t s) {
    hyb_status st = ensure_cap(m, B);
    if (st != HYB_OK) return st;
    const int64_t cap = m->cap;
    k_pack_input<<<(unsigned)((B * m->kin + 255) / 256), 256, 0, s>>>(x, B, m->n_in, m->kin, m->act);
    m->launches++;
    for (int l = 0; l < m->L; l++) {
        const int fi = pad16(layer_in(m, l)), fo = pad16(layer_out(m, l));
        const __nv_bfloat16* X = m->act + (size_t)l * cap * 256;
        float* H = m->pre + (size_t)l * cap * 256;
        // H[B][fo] = X[B][fi] W^T, W stored [fo][fi]
        gemm((int)B, fo, fi, X, 256, 1, m->wbf + m->wb_off[l], 1, fi, H, 256, 0, s, m->launches, m->err);
        const bool hidden = l < m->L - 1;
        k_bias_act<<<(unsigned)((B * fo + 255) / 256), 256, 0, s>>>(H, m->master + m->b_off[l], B, layer_out(m, l), fo, hidden,
                                                                  m->act + (size_t)(l + 1) * cap * 256, y);
        m->launches++;
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

static hyb_status backward(hyb_mlp* m, const float* tgt, int64_t B, cudaStream_t s) {
    const int64_t cap = m->cap;
    HYB_CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    k_loss<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(m->pre + (size_t)(m->L - 1) * cap * 256, tgt, B, m->dh, m->loss);
    m->launches++;
    for (int l = m->L - 1; l >= 0; l--) {
        const int fi = pad16(layer_in(m, l)), fo = pad16(layer_out(m, l));
        const int ni = layer_in(m, l), no = layer_out(m, l);
        k_to_bf16<<<(unsigned)((B * 256 + 255) / 256), 256, 0, s>>>(m->dh, B * 256, m->dhb);
        m->launches++;
        // dW[fo][fi] = dH^T X: M = fo, N = fi, K = B (B padded to 16 with zero rows)
        gemm(fo, fi, (int)B, m->dhb, 1, 256, m->act + (size_t)l * cap * 256, 256, 1, m->dx, 256, 0, s, m->launches, m->err);
        k_copy_grad<<<(no * ni + 255) / 256, 256, 0, s>>>(m->dx, no, ni, 256, m->grad + m->w_off[l]);
        m->launches++;
        k_colsum<<<no, 256, 0, s>>>(m->dh, B, no, m->grad + m->b_off[l]);
        m->launches++;
        if (l > 0) {
            // dX[B][fi] = dH[B][fo] W[fo][fi]
            gemm((int)B, fi, fo, m->dhb, 256, 1, m->wbf + m->wb_off[l], fi, 1, m->dx, 256, 0, s, m->launches, m->err);
            k_act_back<<<(unsigned)((B * fi + 255) / 256), 256, 0, s>>>(m->dx, m->pre + (size_t)(l - 1) * cap * 256, B, ni, fi, m->dh);
            m->launches++;
        }
    }
    HYB_CUDA_TRY(cudaGetLastError());
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" {

hyb_status hyb_mlp_create(int n_in, int width, int depth, const float* init_params, hyb_mlp** out) {
    if (!out || n_in < 1 || n_in > 256 || width < 1 || width > 256 || depth < 1 || depth > 16) {
        set_error("hyb_mlp_create: bad sizes");
        return HYB_EINVAL;
    }
    *out = nullptr;
    hyb_mlp* m = new hyb_mlp();
    m->n_in = n_in; m->width = width; m->depth = depth; m->kin = pad16(n_in); m->L = depth + 1;
    size_t off = 0, woff = 0;
    for (int l = 0; l < m->L; l++) {
        const int fi = layer_in(m, l), fo = layer_out(m, l);
        m->w_off.push_back(off); off += (size_t)fo * fi;
        m->b_off.push_back(off); off += fo;
        m->wb_off.push_back(woff); woff += (size_t)pad16(fo) * pad16(fi);
    }
    m->n_params = off;
    cudaError_t e = cudaMalloc(&m->master, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&m->wbf, sizeof(__nv_bfloat16) * woff);
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
    return forward(m, x, B, y, (cudaStream_t)stream);
}

hyb_status hyb_mlp_gradients(hyb_mlp* m, const float* x, const float* target, int64_t B, float* grad_host, float* loss_host,
                             void* stream) {
    if (!m || !x || !target || B < 1) { set_error("hyb_mlp_gradients: bad arguments"); return HYB_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    hyb_status st = forward(m, x, B, nullptr, s);
    if (st == HYB_OK) st = backward(m, target, B, s);
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
    hyb_status st = forward(m, x, B, nullptr, s);
    if (st == HYB_OK) st = backward(m, target, B, s);
    if (st != HYB_OK) return st;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->master, m->grad, m->adam_m, m->adam_v, (int64_t)m->n_params,
                                                                lr, b1, b2, 1e-8f, c1, c2);
    m->launches++;
    HYB_CUDA_TRY(cudaGetLastError());
    st = refresh(m, s);
    if (st != HYB_OK) return st;
    if (loss_dev) HYB_CUDA_TRY(cudaMemcpyAsync(loss_dev, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return HYB_OK;
}

int64_t hyb_mlp_launch_count(const hyb_mlp* m) { return m ? m->launches : 0; }

hyb_status hyb_mlp_destroy(hyb_mlp* m) {
    if (!m) return HYB_OK;
    cudaDeviceSynchronize();
    cudaFree(m->master); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->grad); cudaFree(m->wbf); cudaFree(m->loss);
    cudaFree(m->err);
    if (m->act) { cudaFree(m->act); cudaFree(m->pre); cudaFree(m->dh); cudaFree(m->dhb); cudaFree(m->dx); }
    delete m;
    return HYB_OK;
}

}  // extern "C"
