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
// fit the array, so any grid size is accepted as long as one row fits.
#include <mutex>
#include <vector>

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

template <typename T>
__global__ void k_noalloc_scale(cplx<T>* __restrict__ spec, int nk, const T* __restrict__ fac) {
    cplx<T>* X = spec + (int64_t)blockIdx.x * nk;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) X[k] = cscale(X[k], fac[k]);
}

template <typename T>
static hyb_status run(const hyb_grid_desc& d, T* j1, cudaStream_t s) {
    using C = cplx<T>;
    const int n1 = d.n1, M = n1 / 2, nk = M + 1;
    const int64_t rows = (int64_t)d.n2 * (d.dims == 3 ? d.n3 : 1);
    // tables in the head of the array: corr[nk], twS[M], twN[M] and, for n1 = 1024, tw8; then row blocks
    auto up16 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t n8 = M == 512 ? (size_t)kTw8 : 0;
    const size_t tab_bytes = up16(sizeof(T) * nk) + up16(sizeof(C) * M) * 2 + up16(sizeof(C) * n8);
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
    C* twS = (C*)(p + up16(sizeof(T) * nk));
    C* twN = (C*)(p + up16(sizeof(T) * nk) + up16(sizeof(C) * M));
    C* tw8 = (C*)(p + up16(sizeof(T) * nk) + 2 * up16(sizeof(C) * M));
    C* spec = (C*)(p + tab_bytes);
    const int64_t rows_per_block = (int64_t)((kNoallocBytes - tab_bytes) / row_bytes);

    // FP64 tables on the host, rounded once (the same quantities hyb_create_grid computes)
    const double pi = 3.14159265358979323846;
    std::vector<T> hc(nk);
    const std::vector<C> hm = stockham_twiddles<C>(M);
    std::vector<C> hn(M);
    const std::vector<C> h8 = n8 ? tw8_table<C>() : std::vector<C>();
    for (int k = 0; k < nk; k++) {
        const double k1 = 2.0 * pi * k / (n1 * d.dx1);
        const double kfd = sin(0.5 * k1 * d.dx1) / (0.5 * d.dx1);
        double ke = k1;
        if (d.yee_mode) ke = kfd;
        else if (d.kmod_max != 0.0) {
            const double kg = 2.0 * pi / d.dx1, kl = d.kmod_l * kg, ku = d.kmod_u * kg, km = 0.5 * (kl + ku);
            if (k1 >= kl && k1 <= ku) { const double c = cos(0.5 * pi * (k1 - km) / (kl - km)); ke += d.kmod_max * kg * c * c; }
        }
        hc[k] = (T)(k == 0 ? 1.0 : kfd / ke);
    }
    for (int j = 0; j < M; j++) {
        const double b = -2.0 * pi * j / n1;
        hn[j] = mkc<C>((T)cos(b), (T)sin(b));
    }
    // pageable source: the copies are staged before cudaMemcpyAsync returns
    HYB_CUDA_TRY(cudaMemcpyAsync(corr, hc.data(), sizeof(T) * nk, cudaMemcpyHostToDevice, s));
    HYB_CUDA_TRY(cudaMemcpyAsync(twS, hm.data(), sizeof(C) * M, cudaMemcpyHostToDevice, s));
    HYB_CUDA_TRY(cudaMemcpyAsync(twN, hn.data(), sizeof(C) * M, cudaMemcpyHostToDevice, s));
    if (n8) HYB_CUDA_TRY(cudaMemcpyAsync(tw8, h8.data(), sizeof(C) * n8, cudaMemcpyHostToDevice, s));
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
        k_noalloc_scale<T><<<(unsigned)nr, 256, 0, s>>>(spec, nk, corr);
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
