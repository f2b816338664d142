// noalloc.cu -- hyb_correct_current_noalloc: the j1 correction of
// hyb_correct_current for callers that cannot allocate device memory.
//
// Some host programs cannot call cudaMalloc at the point where they need the
// correction: their device memory is handed out by a framework's own pool
// (so a stray cudaMalloc can fail or fragment it), or they run a latency-
// critical loop where cudaMalloc's implicit device synchronisation is not
// acceptable.  This entry point therefore allocates nothing: its working
// memory (the per-mode tables and the k1-space copy of a block of rows) is the
// file-scope array g_noalloc_scratch below, which every GPU that loads the
// library holds until the process exits.  Rows are processed in blocks that
// fit the array, so any grid size is accepted as long as one row fits.  The
// tables are computed by a kernel on the call's stream, not copied from the
// host, so a call makes no host-to-device copy and does not block the host on
// the stream.
#include <algorithm>
#include <mutex>

#include "hyb_internal.cuh"

namespace hyb {

// Size of the static working array (bytes); one row's k1-space copy plus the
// tables must fit in it.
constexpr size_t kNoallocBytes = 8u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Host-side addresses of g_noalloc_scratch per device (set up once per device).
constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

static hyb_status noalloc_address(void** out) {
    int dev = 0;
    HYB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal %d out of range", dev); return HYB_EINVAL; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // the device address of the array
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HYB_OK;
}

// The tables of one call, written on the device into the head of the static array (no
// host copies): corr[nk] (Eq. currentcorrection, from the same mode_k the grid tables use),
// twS[M] (stockham_twiddles), twN[M] = W_n1^j and, for n1 = 1024, tw8[kTw8]; FP64, rounded once.
template <typename T>
__global__ void k_noalloc_tables(T* __restrict__ corr, cplx<T>* __restrict__ twS, cplx<T>* __restrict__ twN,
                                 cplx<T>* __restrict__ tw8, int n1, double dx1, int yee_mode, double kmod_l,
                                 double kmod_u, double kmod_max, int n8) {
    using C = cplx<T>;
    const int M = n1 / 2, nk = M + 1;
    const int total = nk + 2 * M + n8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nk) {
            corr[i] = (T)mode_corr(i, mode_k(i, n1, dx1, yee_mode, kmod_l, kmod_u, kmod_max));
            continue;
        }
        int j = i - nk, num, den;
        C* dst;
        if (j < M) { stockham_tw_frac(M, j, &num, &den); dst = twS + j; }
        else if (j < 2 * M) { j -= M; num = j; den = n1; dst = twN + j; }
        else { j -= 2 * M; tw8_frac(j, &num, &den); dst = tw8 + j; }
        double sn, cs;
        sincospi(-2.0 * (double)num / (double)den, &sn, &cs);   // exp(-2 pi i num/den)
        *dst = mkc<C>((T)cs, (T)sn);
    }
}

// X[r][k] *= fac[k] over nr rows of nk modes (grid-stride over all nr * nk entries)
template <typename T>
__global__ void k_noalloc_scale(cplx<T>* __restrict__ spec, int nk, int64_t nr, const T* __restrict__ fac) {
    const int64_t n = nr * nk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        spec[i] = cscale(spec[i], fac[i % nk]);
}

template <typename T>
static hyb_status run(const hyb_grid_desc& d, T* j1, cudaStream_t s) {
    using C = cplx<T>;
    const int n1 = d.n1, M = n1 / 2, nk = M + 1;
    const int64_t rows = (int64_t)d.n2 * (d.dims == 3 ? d.n3 : 1);
    // tables in the head of the array: corr[nk], twS[M], twN[M] and, for n1 = 1024, tw8; then row blocks
    auto up256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int n8 = M == 512 ? kTw8 : 0;
    const size_t tab_bytes = up256(sizeof(T) * nk) + up256(sizeof(C) * M) * 2 + up256(sizeof(C) * n8);
    const size_t row_bytes = sizeof(C) * (size_t)nk;
    if (tab_bytes + row_bytes > kNoallocBytes) {
        set_error("hyb_correct_current_noalloc: n1 = %d needs %zu bytes of working memory, more than the %zu available",
                  n1, tab_bytes + row_bytes, kNoallocBytes);
        return HYB_EINVAL;
    }
    void* base = nullptr;
    hyb_status st = noalloc_address(&base);
    if (st != HYB_OK) return st;
    char* p = (char*)base;
    T* corr = (T*)p;
    C* twS = (C*)(p + up256(sizeof(T) * nk));
    C* twN = (C*)(p + up256(sizeof(T) * nk) + up256(sizeof(C) * M));
    C* tw8 = (C*)(p + up256(sizeof(T) * nk) + 2 * up256(sizeof(C) * M));
    C* spec = (C*)(p + tab_bytes);
    const int64_t rows_per_block = (int64_t)((kNoallocBytes - tab_bytes) / row_bytes);

    // every table entry is rewritten, so an earlier call's tables (other n1, dx1 or mode
    // switches) leave nothing behind; stream-ordered before the transforms that read them
    {
        const int total = nk + 2 * M + n8;
        k_noalloc_tables<T><<<(total + 255) / 256, 256, 0, s>>>(corr, twS, twN, tw8, n1, d.dx1, d.yee_mode, d.kmod_l,
                                                               d.kmod_u, d.kmod_max, n8);
        HYB_CUDA_TRY(cudaGetLastError());
    }
    ModeTables<T> t;
    t.twS = twS;
    t.twN = twN;
    t.tw8 = n8 ? tw8 : nullptr;
    // the row blocks are overwritten completely by the forward transform, so
    // nothing left by an earlier call needs clearing
    for (int64_t r0 = 0; r0 < rows; r0 += rows_per_block) {
        const int64_t nr = (rows - r0 < rows_per_block) ? rows - r0 : rows_per_block;
        T* rowp = j1 + r0 * n1;
        HYB_CUDA_TRY((rfft_rows<T, T>(rowp, spec, n1, nr, t, s)));
        const int64_t n = nr * nk;
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
        k_noalloc_scale<T><<<blocks, 256, 0, s>>>(spec, nk, nr, corr);
        HYB_CUDA_TRY(cudaGetLastError());
        HYB_CUDA_TRY((irfft_rows<T, T>(spec, rowp, n1, nr, t, s)));
    }
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" hyb_status hyb_correct_current_noalloc(const hyb_grid_desc* desc, void* j1, void* stream) {
    if (!desc || !j1) { set_error("hyb_correct_current_noalloc: null argument"); return HYB_EINVAL; }
    const hyb_grid_desc& d = *desc;
    if (d.dims != 2 && d.dims != 3) { set_error("dims must be 2 or 3"); return HYB_EINVAL; }
    if (d.n1 < 8 || d.n1 > 8192 || (d.n1 & (d.n1 - 1))) { set_error("n1 must be a power of two in [8, 8192]"); return HYB_EINVAL; }
    if (d.n2 < 1 || (d.dims == 3 && d.n3 < 1)) { set_error("bad n2/n3"); return HYB_EINVAL; }
    if (!(d.dx1 > 0)) { set_error("dx1 must be positive"); return HYB_EINVAL; }
    if (((uintptr_t)j1 & 15u) != 0) { set_error("j1 not 16-byte aligned"); return HYB_EALIGN; }
    if (d.precision == 32) return run<float>(d, (float*)j1, (cudaStream_t)stream);
    if (d.precision == 64) return run<double>(d, (double*)j1, (cudaStream_t)stream);
    set_error("precision must be 32 or 64");
    return HYB_EINVAL;
}
