// hyb_api.cu -- C ABI of libhyb.so (declared in include/hyb.h): validation,
// FP64 host computation of the per-mode tables, scratch ownership and
// dispatch to the three-pass or fused advance.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "hyb_internal.cuh"
#include "batch_step.cuh"
#include "fused_api.cuh"

namespace hyb {

int resident_grid(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, int> cache;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, kernel, smem * 4096 + (size_t)threads);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    const int r = sms * occ > 0 ? sms * occ : 1;
    cache[key] = r;
    return r;
}

cudaError_t func_attr_once(const void* kernel, cudaFuncAttribute attr, int value) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int>, int> done;   // value set per (device, kernel, attribute)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, kernel, (int)attr);
    const auto it = done.find(key);
    if (it != done.end() && it->second == value) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, attr, value);
    if (e == cudaSuccess) done[key] = value;
    return e;
}

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

hyb_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HYB_ENOMEM : HYB_ECUDA;
}

static const double kPi = 3.14159265358979323846;

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Sec. 2.2: dt <= 2 / sqrt(pi^2/dx1^2 + 4/dx2^2 [+ 4/dx3^2]).  Quasi-3D mode m:
// the (i m / r) terms raise the radial operator's largest eigenvalue to at
// most (4 m^2 + 6)/dr^2 (it sits at the axis), so 4/dx2^2 becomes (4 m^2 + 6)/dx2^2.
static double courant_limit(const hyb_grid_desc& d) {
    double s = kPi * kPi / (d.dx1 * d.dx1);
    if (d.dims == 20) s += (4.0 * d.azimuthal_m * d.azimuthal_m + 6.0) / (d.dx2 * d.dx2);
    else s += 4.0 / (d.dx2 * d.dx2);
    if (d.dims == 3) s += 4.0 / (d.dx3 * d.dx3);
    return 2.0 / sqrt(s);
}

// FP64 per-mode quantities for kappa = 0..n1/2
struct HostModes {
    std::vector<double> keff, corr, filt, sgp_re, sgp_im;
};

static HostModes host_modes(const hyb_grid_desc& d) {
    const int M = d.n1 / 2;
    HostModes h;
    h.keff.resize(M + 1); h.corr.resize(M + 1); h.filt.resize(M + 1);
    h.sgp_re.resize(M + 1); h.sgp_im.resize(M + 1);
    const double kn = kPi / d.dx1;
    const bool filt_on = d.filt_kc > 0.0 && d.filt_kc < 1.0;
    for (int k = 0; k <= M; k++) {
        const ModeK mk = mode_k(k, d.n1, d.dx1, d.yee_mode, d.kmod_l, d.kmod_u, d.kmod_max);
        const double k1 = mk.k1, ke = mk.keff;                           // hybrid: [k]1 -> k1 (or Yee, or bump)
        h.keff[k] = ke;
        h.corr[k] = mode_corr(k, mk);                                    // Eq. currentcorrection
        double f = 1.0;
        if (filt_on) {
            const double kc = d.filt_kc * kn, w = d.filt_w * kn, a = fabs(k1);
            if (w <= 0.0) f = a <= kc ? 1.0 : 0.0;
            else if (a <= kc - 0.5 * w) f = 1.0;
            else if (a >= kc + 0.5 * w) f = 0.0;
            else { const double c = cos(0.5 * kPi * (a - kc + 0.5 * w) / w); f = c * c; }
        }
        h.filt[k] = f;
        const double ph = 0.5 * k1 * d.dx1;                              // half-cell shift
        h.sgp_re[k] = -ke * sin(ph);                                      // i ke exp(+i ph)
        h.sgp_im[k] = ke * cos(ph);
    }
    return h;
}

template <typename T>
static hyb_status upload_tables(hyb_grid* g, const HostModes& h, ModeTables<T>& t) {
    using C = cplx<T>;
    const hyb_grid_desc& d = g->d;
    const int M = d.n1 / 2, nk = M + 1;
    const double dt = d.dt, A = d.ampere;
    std::vector<C> S(nk), sgp(nk), twM(M), twN(M);
    std::vector<T> cj1(nk), cj(nk), corr(nk), filt(nk);
    for (int k = 0; k < nk; k++) {
        S[k] = mkc<C>((T)(dt * h.sgp_re[k]), (T)(dt * h.sgp_im[k]));
        sgp[k] = mkc<C>((T)h.sgp_re[k], (T)h.sgp_im[k]);
        const double c1 = d.correct_j1 ? h.corr[k] : 1.0;
        cj1[k] = (T)(A * dt * h.filt[k] * c1);
        cj[k] = (T)(A * dt * h.filt[k]);
        corr[k] = (T)h.corr[k];
        filt[k] = (T)h.filt[k];
    }
    for (int j = 0; j < M; j++) {
        const double a = -2.0 * kPi * (double)j / (double)M;
        twM[j] = mkc<C>((T)cos(a), (T)sin(a));
        const double b = -2.0 * kPi * (double)j / (double)d.n1;
        twN[j] = mkc<C>((T)cos(b), (T)sin(b));
    }
    const std::vector<C> tw8 = M == 512 ? tw8_table<C>() : std::vector<C>();
    const std::vector<C> twS = stockham_twiddles<C>(M);
    const size_t bytes = sizeof(C) * (4 * (size_t)nk + 3 * (size_t)M + tw8.size()) + sizeof(T) * 4 * (size_t)nk + 256;
    char* base = nullptr;
    HYB_CUDA_TRY(cudaMalloc(&base, bytes));
    char* p = base;
    auto take = [&](size_t n) { char* r = p; p += (n + 15) & ~(size_t)15; return r; };
    t.S = (C*)take(sizeof(C) * nk);
    t.sgp = (C*)take(sizeof(C) * nk);
    t.twM = (C*)take(sizeof(C) * M);
    t.twN = (C*)take(sizeof(C) * M);
    t.cj1 = (T*)take(sizeof(T) * nk);
    t.cj = (T*)take(sizeof(T) * nk);
    t.corr = (T*)take(sizeof(T) * nk);
    t.filt = (T*)take(sizeof(T) * nk);
    if (!tw8.empty()) t.tw8 = (C*)take(sizeof(C) * tw8.size());
    t.twS = (C*)take(sizeof(C) * M);
    HYB_CUDA_TRY(cudaMemcpy(t.S, S.data(), sizeof(C) * nk, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.sgp, sgp.data(), sizeof(C) * nk, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.twM, twM.data(), sizeof(C) * M, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.twN, twN.data(), sizeof(C) * M, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.cj1, cj1.data(), sizeof(T) * nk, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.cj, cj.data(), sizeof(T) * nk, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.corr, corr.data(), sizeof(T) * nk, cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.filt, filt.data(), sizeof(T) * nk, cudaMemcpyHostToDevice));
    if (!tw8.empty()) HYB_CUDA_TRY(cudaMemcpy(t.tw8, tw8.data(), sizeof(C) * tw8.size(), cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMemcpy(t.twS, twS.data(), sizeof(C) * M, cudaMemcpyHostToDevice));
    return HYB_OK;
}

static void free_tables_f(ModeTables<float>& t) { if (t.S) cudaFree(t.S); t = ModeTables<float>(); }
static void free_tables_d(ModeTables<double>& t) { if (t.S) cudaFree(t.S); t = ModeTables<double>(); }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace hyb

using namespace hyb;

extern "C" {

const char* hyb_last_error(void) { return hyb::g_err; }

double hyb_courant_limit(const hyb_grid_desc* desc) {
    if (!desc) return 0.0;
    return courant_limit(*desc);
}

hyb_status hyb_create_grid(const hyb_grid_desc* desc, void* stream, hyb_grid** out) {
    set_error("");
    if (!desc || !out) { set_error("hyb_create_grid: null argument"); return HYB_EINVAL; }
    *out = nullptr;
    hyb_grid_desc d = *desc;
    if (d.dims != 2 && d.dims != 3 && d.dims != 20) { set_error("dims must be 2, 3 or 20 (got %d)", d.dims); return HYB_EINVAL; }
    if (d.dims != 3) { d.n3 = 1; d.dx3 = d.dx3 > 0 ? d.dx3 : 1.0; }
    if (d.dims == 20 && (d.azimuthal_m < 0 || d.azimuthal_m > 64)) { set_error("azimuthal_m must be in [0, 64]"); return HYB_EINVAL; }
    if (d.dims == 20 && d.n2 > 65535) { set_error("quasi-3D grids take at most 65535 radial rows (got %d)", d.n2); return HYB_EINVAL; }
    if (!is_pow2(d.n1) || d.n1 < 8 || d.n1 > 8192) { set_error("n1 must be a power of two in [8, 8192] (got %d)", d.n1); return HYB_EINVAL; }
    if (d.n2 < 2 || (d.dims == 3 && d.n3 < 2)) { set_error("n2 (and n3 in 3D) must be >= 2"); return HYB_EINVAL; }
    if ((int64_t)d.n2 * d.n3 > (int64_t)1 << 30) { set_error("too many rows"); return HYB_EINVAL; }
    if (!(d.dx1 > 0 && d.dx2 > 0 && (d.dims == 2 || d.dx3 > 0) && d.dt > 0)) { set_error("cell sizes and dt must be positive"); return HYB_EINVAL; }
    if (d.precision != 32 && d.precision != 64) { set_error("precision must be 32 or 64 (got %d)", d.precision); return HYB_EINVAL; }
    if (d.ampere == 0.0) d.ampere = 4.0 * kPi;
    const double cl = courant_limit(d);
    if (d.dt > cl * (1.0 + 1e-12)) {
        set_error("dt = %.17g exceeds the Courant limit %.17g of the hybrid solver", d.dt, cl);
        return HYB_ECOURANT;
    }
    if (d.path < 0 || d.path > 4) { set_error("path must be 0, 1, 2, 3 or 4"); return HYB_EINVAL; }
    if (d.path >= 3 && !(d.precision == 32 && d.dims != 20 && d.n1 >= 16 && d.n1 <= 1024)) {
        set_error("paths 3 and 4 (DFT-GEMM) need precision 32, dims 2 or 3 and 16 <= n1 <= 1024");
        return HYB_EINVAL;
    }
    const bool fused_ok = d.dims != 20 && fused_supported(d);
    if (d.dims == 20 && d.path == 2) { set_error("quasi-3D grids run the three-pass path"); return HYB_EINVAL; }
    if (d.path == 2 && !fused_ok) {
        set_error("fused path needs precision 32, dims 2, n1 in [512, 4096] and n2 >= 4");
        return HYB_EINVAL;
    }
    hyb_grid* g = new hyb_grid();
    g->d = d;
    g->stream = (cudaStream_t)stream;
    // auto: the fused single pass where it applies; otherwise the three-pass advance with the
    // radix FFT, which measured faster on GB300 than the DFT-GEMM (path 3) at every n1 from 16 to 1024
    g->path = (d.path == 0) ? (fused_ok ? 2 : 1) : d.path;
    g->rows = (int64_t)d.n2 * d.n3;
    g->cells = g->rows * d.n1;
    g->nk = d.n1 / 2 + 1;
    hyb_status st = HYB_OK;
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) { st = cuda_fail(ce, "cudaGetDevice"); hyb_destroy_grid(g); return st; }
    HostModes h = host_modes(d);
    st = upload_tables<double>(g, h, g->td);
    if (st == HYB_OK && d.precision == 32) st = upload_tables<float>(g, h, g->tf);
    if (st == HYB_OK) {
        ce = cudaMalloc(&g->diag_acc, 16 * sizeof(double));
        if (ce == cudaSuccess) ce = cudaMalloc(&g->dflag, sizeof(int));
        if (ce == cudaSuccess) ce = cudaMemset(g->dflag, 0, sizeof(int));
        if (ce != cudaSuccess) st = cuda_fail(ce, "cudaMalloc(accumulators)");
    }
    if (st == HYB_OK && d.dims == 20) st = quasi3d_create(g);
    if (st == HYB_OK && d.dims != 20) {
        const size_t csz = d.precision == 32 ? sizeof(float2) : sizeof(double2);
        const int nf = g->path == 2 ? 3 : 9;
        g->spec_fields = nf;
        g->spec_bytes = (size_t)nf * g->rows * g->nk * csz;
        ce = cudaMalloc(&g->spec, g->spec_bytes);
        if (ce != cudaSuccess) { g->spec = nullptr; st = cuda_fail(ce, "cudaMalloc(spectral scratch)"); }
    }
    if (st == HYB_OK && g->path == 2) st = fused_create(g);
    if (st == HYB_OK && g->path >= 3) st = dftgemm_create(g);
    if (st != HYB_OK) { hyb_destroy_grid(g); return st; }
    *out = g;
    return HYB_OK;
}

hyb_status hyb_set_resident(hyb_grid* g, int on) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (on != 0 && on != 1) { set_error("hyb_set_resident: on must be 0 or 1"); return HYB_EINVAL; }
    if (on && g->d.dims == 20) { set_error("hyb_set_resident: quasi-3D grids keep no k1-resident state"); return HYB_EINVAL; }
    if (on && g->spec_fields < 9) {
        // a fused-path grid keeps only j's spectra: room for E, B too
        const size_t csz = g->d.precision == 32 ? sizeof(float2) : sizeof(double2);
        const size_t bytes = (size_t)9 * g->rows * g->nk * csz;
        void* p = nullptr;
        HYB_CUDA_TRY(cudaStreamSynchronize(g->stream));
        HYB_CUDA_TRY(cudaMalloc(&p, bytes));
        if (g->spec) cudaFree(g->spec);
        g->spec = p;
        g->spec_bytes = bytes;
        g->spec_fields = 9;
    }
    g->resident = on != 0;
    g->res_stale = true;
    g->step_dirty = true;
    return HYB_OK;
}

hyb_status hyb_set_stream(hyb_grid* g, void* stream) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    g->stream = (cudaStream_t)stream;
    return HYB_OK;
}

hyb_status hyb_bind_fields(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3], void* rho) {
    if (!g || !E || !B || !J) { set_error("hyb_bind_fields: null argument"); return HYB_EINVAL; }
    g->step_dirty = true;
    for (int c = 0; c < 3; c++) {
        if (!E[c] || !B[c] || !J[c]) { set_error("hyb_bind_fields: null field pointer"); return HYB_EINVAL; }
        if (!aligned16(E[c]) || !aligned16(B[c]) || !aligned16(J[c])) { set_error("hyb_bind_fields: field not 16-byte aligned"); return HYB_EALIGN; }
    }
    if (rho && !aligned16(rho)) { set_error("hyb_bind_fields: rho not 16-byte aligned"); return HYB_EALIGN; }
    for (int c = 0; c < 3; c++) { g->E[c] = E[c]; g->B[c] = B[c]; g->J[c] = J[c]; }
    g->rho = rho;
    g->bound = true;
    g->res_stale = true;
    return HYB_OK;
}

hyb_status hyb_deposit(hyb_grid* g, const int32_t* cell, const void* off_old, const void* off_new,
                       const void* v3, const void* q, int64_t np, int shape_order) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (!g->bound) { set_error("hyb_deposit: fields not bound"); return HYB_ESTATE; }
    if (np < 0 || shape_order < 1 || shape_order > 3) { set_error("hyb_deposit: bad np or shape_order"); return HYB_EINVAL; }
    if (np > 0 && (!cell || !off_old || !off_new || !q)) { set_error("hyb_deposit: null particle array"); return HYB_EINVAL; }
    if (g->d.dims == 20) { set_error("hyb_deposit: quasi-3D grids take their current from the caller"); return HYB_EINVAL; }
    if (g->d.precision == 32)
        return deposit<float>(g, cell, (const float*)off_old, (const float*)off_new, (const float*)v3, (const float*)q, np, shape_order);
    return deposit<double>(g, cell, (const double*)off_old, (const double*)off_new, (const double*)v3, (const double*)q, np, shape_order);
}

hyb_status hyb_push(hyb_grid* g, int32_t* cell, void* off, void* u, const void* qm, void* off_new, void* v3,
                    int64_t np, int shape_order) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (!g->bound) { set_error("hyb_push: fields not bound"); return HYB_ESTATE; }
    if (np < 0 || shape_order < 1 || shape_order > 3) { set_error("hyb_push: bad np or shape_order"); return HYB_EINVAL; }
    if (np > 0 && (!cell || !off || !u || !qm || !off_new)) { set_error("hyb_push: null particle array"); return HYB_EINVAL; }
    if (g->d.dims == 20) { set_error("hyb_push: quasi-3D grids carry no particles"); return HYB_EINVAL; }
    const size_t real = g->d.precision == 32 ? 4 : 8;
    if (g->d.dims == 2 && ((uintptr_t)cell % 8 || (uintptr_t)off % (2 * real) || (uintptr_t)off_new % (2 * real))) {
        set_error("hyb_push: 2D cell (8 bytes) and off, off_new (2 reals) must be aligned to one particle's pair");
        return HYB_EALIGN;
    }
    if (g->d.precision == 32)
        return push<float>(g, cell, (float*)off, (float*)u, (const float*)qm, (float*)off_new, (float*)v3, np, shape_order);
    return push<double>(g, cell, (double*)off, (double*)u, (const double*)qm, (double*)off_new, (double*)v3, np, shape_order);
}

hyb_status hyb_correct_current(hyb_grid* g) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (!g->bound) { set_error("fields not bound"); return HYB_ESTATE; }
    if (g->d.dims == 20) { set_error("quasi-3D grids apply the correction inside hyb_advance only"); return HYB_EINVAL; }
    return g->d.precision == 32 ? generic_process_current<float>(g, true, false) : generic_process_current<double>(g, true, false);
}

hyb_status hyb_filter(hyb_grid* g) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (!g->bound) { set_error("fields not bound"); return HYB_ESTATE; }
    if (g->d.dims == 20) { set_error("quasi-3D grids apply the filter inside hyb_advance only"); return HYB_EINVAL; }
    return g->d.precision == 32 ? generic_process_current<float>(g, false, true) : generic_process_current<double>(g, false, true);
}

// one step of the three-pass or quasi-3D path enqueued on g->stream
static hyb_status step_once(hyb_grid* g) {
    if (g->d.dims == 20) return quasi3d_advance(g, 1);
    return g->d.precision == 32 ? generic_advance<float>(g, 1) : generic_advance<double>(g, 1);
}

// captures one step on a private stream (launches only: the step's kernels read and write the
// bound arrays and the grid's scratch) into g->step_exec
static hyb_status capture_step(hyb_grid* g) {
    if (g->step_exec) { cudaGraphExecDestroy(g->step_exec); g->step_exec = nullptr; }
    cudaStream_t cs = nullptr;
    HYB_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = g->stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    hyb_status st = HYB_OK;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) {
        g->stream = cs;
        st = step_once(g);
        g->stream = keep;
        e = cudaStreamEndCapture(cs, &graph);
    }
    cudaStreamDestroy(cs);
    if (st != HYB_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "step capture"); }
    e = cudaGraphInstantiate(&g->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { g->step_exec = nullptr; return cuda_fail(e, "step graph instantiation"); }
    g->step_dirty = false;
    return HYB_OK;
}

hyb_status hyb_advance(hyb_grid* g, int nsteps) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if (!g->bound) { set_error("hyb_advance: fields not bound"); return HYB_ESTATE; }
    if (nsteps < 0) { set_error("nsteps < 0"); return HYB_EINVAL; }
    if (nsteps == 0) return HYB_OK;
    if (g->path == 2 && !g->resident) return fused_advance(g, nsteps);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HYB_CUDA_TRY(cudaStreamIsCapturing(g->stream, &cap));
    if (g->resident && g->res_stale && cap == cudaStreamCaptureStatusNone && !g->ev_start) {
        // the importing step (E, B transformed too) runs as plain launches; the step graph
        // captured afterwards is the resident one
        hyb_status st = step_once(g);
        if (st != HYB_OK) return st;
        if (--nsteps == 0) return HYB_OK;
    }
    if (g->ev_start || cap != cudaStreamCaptureStatusNone) {
        // per-step kernel events requested, or the caller is capturing its own graph: plain launches
        for (int s = 0; s < nsteps; s++) {
            hyb_status st = step_once(g);
            if (st != HYB_OK) return st;
        }
        return HYB_OK;
    }
    if (g->step_dirty || !g->step_exec) {
        hyb_status st = capture_step(g);
        if (st != HYB_OK) return st;
    }
    for (int s = 0; s < nsteps; s++) HYB_CUDA_TRY(cudaGraphLaunch(g->step_exec, g->stream));
    return HYB_OK;
}

hyb_status hyb_advance_host(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3], int nsteps) {
    if (!g || !E || !B || !J) { set_error("hyb_advance_host: null argument"); return HYB_EINVAL; }
    if (!g->bound) { set_error("hyb_advance_host: device fields not bound"); return HYB_ESTATE; }
    for (int c = 0; c < 3; c++)
        if (!E[c] || !B[c] || !J[c]) { set_error("hyb_advance_host: null field pointer"); return HYB_EINVAL; }
    if (g->resident) g->res_stale = true;      // E, B come from the host arrays
    if (g->path == 2 && nsteps == 1 && !g->resident) {
        // one fused step: copies in, compute and copies out pipelined over chunks of rows
        hyb_status st = fused_host_advance(g, E, B, J);
        if (st != HYB_OK) return st;
        HYB_CUDA_TRY(cudaStreamSynchronize(g->stream));
        return HYB_OK;
    }
    const size_t bytes = (size_t)g->cells * (g->d.precision == 32 ? 4 : 8) * (g->d.dims == 20 ? 2 : 1);
    for (int c = 0; c < 3; c++) {
        HYB_CUDA_TRY(cudaMemcpyAsync(g->E[c], E[c], bytes, cudaMemcpyHostToDevice, g->stream));
        HYB_CUDA_TRY(cudaMemcpyAsync(g->B[c], B[c], bytes, cudaMemcpyHostToDevice, g->stream));
        HYB_CUDA_TRY(cudaMemcpyAsync(g->J[c], J[c], bytes, cudaMemcpyHostToDevice, g->stream));
    }
    hyb_status st = hyb_advance(g, nsteps);
    if (st != HYB_OK) return st;
    for (int c = 0; c < 3; c++) {
        HYB_CUDA_TRY(cudaMemcpyAsync(E[c], g->E[c], bytes, cudaMemcpyDeviceToHost, g->stream));
        HYB_CUDA_TRY(cudaMemcpyAsync(B[c], g->B[c], bytes, cudaMemcpyDeviceToHost, g->stream));
    }
    HYB_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return HYB_OK;
}

hyb_status hyb_diag(hyb_grid* g, double out[9]) {
    if (!g || !out) { set_error("null argument"); return HYB_EINVAL; }
    if (!g->bound) { set_error("fields not bound"); return HYB_ESTATE; }
    if (g->d.dims == 20) { set_error("hyb_diag: not available for quasi-3D grids"); return HYB_EINVAL; }
    return g->d.precision == 32 ? diag<float>(g, out) : diag<double>(g, out);
}

hyb_status hyb_check(hyb_grid* g) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    int h = 0;
    HYB_CUDA_TRY(cudaStreamSynchronize(g->stream));
    HYB_CUDA_TRY(cudaMemcpy(&h, g->dflag, sizeof(int), cudaMemcpyDeviceToHost));
    HYB_CUDA_TRY(cudaMemset(g->dflag, 0, sizeof(int)));
    if (h & 1) { set_error("hyb_deposit skipped particles outside the documented offset ranges"); return HYB_EDATA; }
    if (h & 2) { set_error("a bounded device-side wait gave up"); return HYB_ETIMEOUT; }
    return HYB_OK;
}

hyb_status hyb_wait_selftest(int which, double seconds, void* stream) {
    if (which < 0 || which > 2 || !(seconds > 0.0 && seconds <= 10.0)) {
        set_error("hyb_wait_selftest: which must be 0, 1 or 2 and seconds in (0, 10]");
        return HYB_EINVAL;
    }
    int dev = 0, khz = 0;
    HYB_CUDA_TRY(cudaGetDevice(&dev));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    int* d = nullptr;
    HYB_CUDA_TRY(cudaMalloc(&d, 3 * sizeof(int)));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(int), s);
    const long long limit = (long long)(seconds * 1e3 * (double)khz);
    if (e == cudaSuccess)
        e = which == 2 ? role_probe(reinterpret_cast<unsigned*>(d), d + 2, limit, s) : wait_probe(d, d + 2, limit, which, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "hyb_wait_selftest");
    if (h & 2) { set_error("a bounded device-side wait gave up"); return HYB_ETIMEOUT; }
    return HYB_OK;
}

hyb_status hyb_destroy_grid(hyb_grid* g) {
    if (!g) return HYB_OK;
    if (g->stream) cudaStreamSynchronize(g->stream); else cudaDeviceSynchronize();
    if (g->step_exec) cudaGraphExecDestroy(g->step_exec);
    if (g->fused) fused_destroy(g);
    if (g->qtab) quasi3d_destroy(g);
    if (g->dft) dftgemm_destroy(g);
    free_tables_f(g->tf);
    free_tables_d(g->td);
    if (g->spec) cudaFree(g->spec);
    if (g->diag_work) cudaFree(g->diag_work);
    if (g->diag_acc) cudaFree(g->diag_acc);
    if (g->dflag) cudaFree(g->dflag);
    delete g;
    return HYB_OK;
}

hyb_status hyb_set_kernel_events(hyb_grid* g, void* start, void* stop) {
    if (!g) { set_error("null grid"); return HYB_EINVAL; }
    if ((start == nullptr) != (stop == nullptr)) { set_error("set both events or neither"); return HYB_EINVAL; }
    g->ev_start = (cudaEvent_t)start;
    g->ev_stop = (cudaEvent_t)stop;
    return HYB_OK;
}

int hyb_grid_path(const hyb_grid* g) { return g ? g->path : 0; }

const char* hyb_step_kernel(const hyb_grid* g) {
    if (!g) return "";
    if (g->resident) return g->path >= 3 ? "k1-resident dft-gemm three-pass step" : "k1-resident three-pass step";
    if (g->path == 2) return fused_step_kernel(g);
    if (g->path >= 3) return g->path == 3 ? "dft-gemm three-pass step (k_dft_tc, 2 parts)"
                                          : "dft-gemm three-pass step (k_dft_tc, 3 parts)";
    return g->d.dims == 20 ? "quasi-3D step" : "three-pass step";
}

int hyb_launches_per_step(const hyb_grid* g) {
    if (!g) return 0;
    if (g->path == 2 && !g->resident) return fused_launches_per_step(g);
    if (g->path >= 3) return 4;      // forward product, Faraday, Ampere, inverse product
    return generic_launches_per_step(g);
}

}  // extern "C"
