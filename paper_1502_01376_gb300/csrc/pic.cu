// pic.cu -- the particle-in-cell loop around the hybrid field advance: the
// time level of each quantity follows the leapfrog of Sec. 2.1 (E at integer
// steps, B at half steps) and the particle step the NCI analysis of the
// Appendix assumes (fields gathered at the particles' time level n with B
// time-centred, the charge-conserving current of Sec. 2.3 from x^n -> x^{n+1}).
//
// One step, with E = E^n, B = B^{n-1/2} bound to the grid and the particles at
// x^n (cell, off) with u^{n-1/2}:
//   1. B^{n+1/2} = B^{n-1/2} + Faraday(E^n): a copy of E and B is advanced one
//      step by a second grid of the same description with zero current (its E
//      is discarded); then B^n = (B^{n-1/2} + B^{n+1/2}) / 2 in that copy;
//   2. gather E^n, B^n and Boris push: u^{n+1/2}, x^{n+1} (hyb_push);
//   3. deposit j^{n+1/2} from x^n -> x^{n+1} (hyb_deposit);
//   4. the hybrid advance: E^{n+1}, B^{n+1/2} (hyb_advance);
//   5. x^{n+1} becomes the next step's x^n (off <- off_new).
// With k1-resident fields (hyb_set_resident) step 1 needs no second grid: B^n =
// B^{n-1/2} + Faraday(E^n)/2 is formed mode by mode from the resident spectra and
// transformed back into scratch arrays, and step 4 transforms only j forward, so a
// step takes 12 row transforms (3 for B^n, 3 for j, 6 for E, B) instead of two
// full advances (30) and the copies of E and B.
#include "hyb_internal.cuh"

struct hyb_pic {
    hyb_grid* g = nullptr;        // the caller's grid (borrowed)
    hyb_grid* shadow = nullptr;   // the same description, bound to the scratch copy and zero current
    void* scratch = nullptr;      // E'[3], B'[3], J'[3] = 0
    size_t field_bytes = 0;
    // one step captured as a CUDA graph, replayed for the later steps of a call (and of later calls
    // with the same arguments): its own stream, fork/join events, and the arguments it was taken with
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* key[12] = {};
    int64_t key_np = -1;
    int key_order = 0, key_path = 0;
    bool key_res = false;
};

namespace hyb {

constexpr int kPicGraphMinSteps = 4;   // calls of at least this many steps replay a captured step

// B'[c] <- (B'[c] + B[c]) / 2 over the three components
template <typename T>
__global__ void k_time_centre(T* __restrict__ b0, T* __restrict__ b1, T* __restrict__ b2, const T* __restrict__ a0,
                              const T* __restrict__ a1, const T* __restrict__ a2, int64_t cells) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * cells; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / cells);
        const int64_t k = i - c * cells;
        T* b = c == 0 ? b0 : c == 1 ? b1 : b2;
        const T* a = c == 0 ? a0 : c == 1 ? a1 : a2;
        b[k] = (T)0.5 * (b[k] + a[k]);
    }
}

template <typename T>
static hyb_status pic_step(hyb_pic* p, int32_t* cell, T* off, T* u, const T* qm, const T* q, T* off_new, T* v3,
                           int64_t np, int order) {
    hyb_grid* g = p->g;
    if (g->resident) {
        void* Bh[3];
        for (int c = 0; c < 3; c++) Bh[c] = (char*)p->scratch + (size_t)(3 + c) * p->field_bytes;
        hyb_status st = HYB_OK;
        if (g->res_stale) st = generic_resident_import<T>(g);                  // E^n, B^{n-1/2} spectra
        if (st == HYB_OK) st = generic_b_half<T>(g, Bh);                        // B^n
        if (st == HYB_OK) st = push_fields<T>(g, g->E, Bh, cell, off, u, qm, off_new, v3, np, order);
        if (st == HYB_OK) st = hyb_deposit(g, cell, off, off_new, v3, q, np, order);
        if (st == HYB_OK) st = hyb_advance(g, 1);                               // j forward only
        if (st != HYB_OK) return st;
        if (np > 0)
            HYB_CUDA_TRY(cudaMemcpyAsync(off, off_new, sizeof(T) * (size_t)np * g->d.dims, cudaMemcpyDeviceToDevice, g->stream));
        return HYB_OK;
    }
    hyb_grid* s = p->shadow;
    s->stream = g->stream;
    char* base = (char*)p->scratch;
    void* Es[3];
    void* Bs[3];
    for (int c = 0; c < 3; c++) {
        Es[c] = base + (size_t)c * p->field_bytes;
        Bs[c] = base + (size_t)(3 + c) * p->field_bytes;
        HYB_CUDA_TRY(cudaMemcpyAsync(Es[c], g->E[c], p->field_bytes, cudaMemcpyDeviceToDevice, g->stream));
        HYB_CUDA_TRY(cudaMemcpyAsync(Bs[c], g->B[c], p->field_bytes, cudaMemcpyDeviceToDevice, g->stream));
    }
    hyb_status st = hyb_advance(s, 1);                           // B' = B^{n+1/2}
    if (st != HYB_OK) return st;
    {
        const int64_t n = 3 * g->cells;
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
        k_time_centre<T><<<blocks, 256, 0, g->stream>>>((T*)Bs[0], (T*)Bs[1], (T*)Bs[2], (const T*)g->B[0],
                                                        (const T*)g->B[1], (const T*)g->B[2], g->cells);
        HYB_CUDA_TRY(cudaGetLastError());
    }
    st = push_fields<T>(g, g->E, Bs, cell, off, u, qm, off_new, v3, np, order);   // u^{n+1/2}, x^{n+1}
    if (st != HYB_OK) return st;
    st = hyb_deposit(g, cell, off, off_new, v3, q, np, order);  // j^{n+1/2}
    if (st != HYB_OK) return st;
    st = hyb_advance(g, 1);                                      // E^{n+1}, B^{n+1/2}
    if (st != HYB_OK) return st;
    const int dims = g->d.dims;
    if (np > 0) HYB_CUDA_TRY(cudaMemcpyAsync(off, off_new, sizeof(T) * (size_t)np * dims, cudaMemcpyDeviceToDevice, g->stream));
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" {

hyb_status hyb_pic_create(hyb_grid* g, hyb_pic** out) {
    if (!g || !out) { set_error("hyb_pic_create: null argument"); return HYB_EINVAL; }
    *out = nullptr;
    if (!g->bound) { set_error("hyb_pic_create: fields not bound"); return HYB_ESTATE; }
    if (g->d.dims == 20) { set_error("hyb_pic_create: quasi-3D grids carry no particles"); return HYB_EINVAL; }
    hyb_pic* p = new hyb_pic();
    p->g = g;
    p->field_bytes = (size_t)g->cells * (g->d.precision == 32 ? 4 : 8);
    cudaError_t e = cudaMalloc(&p->scratch, 9 * p->field_bytes);
    if (e != cudaSuccess) { p->scratch = nullptr; hyb_pic_destroy(p); return cuda_fail(e, "cudaMalloc(pic scratch)"); }
    e = cudaMemset((char*)p->scratch + 6 * p->field_bytes, 0, 3 * p->field_bytes);
    if (e != cudaSuccess) { hyb_pic_destroy(p); return cuda_fail(e, "cudaMemset(pic scratch)"); }
    hyb_grid_desc d = g->d;
    d.path = g->path;
    hyb_status st = hyb_create_grid(&d, g->stream, &p->shadow);
    if (st != HYB_OK) { p->shadow = nullptr; hyb_pic_destroy(p); return st; }
    void* E[3];
    void* B[3];
    void* J[3];
    for (int c = 0; c < 3; c++) {
        E[c] = (char*)p->scratch + (size_t)c * p->field_bytes;
        B[c] = (char*)p->scratch + (size_t)(3 + c) * p->field_bytes;
        J[c] = (char*)p->scratch + (size_t)(6 + c) * p->field_bytes;
    }
    st = hyb_bind_fields(p->shadow, E, B, J, nullptr);
    if (st != HYB_OK) { hyb_pic_destroy(p); return st; }
    *out = p;
    return HYB_OK;
}

hyb_status hyb_pic_step(hyb_pic* p, int32_t* cell, void* off, void* u, const void* qm, const void* q, void* off_new,
                        void* v3, int64_t np, int shape_order, int nsteps) {
    if (!p) { set_error("hyb_pic_step: null pic"); return HYB_EINVAL; }
    if (nsteps < 0 || np < 0 || shape_order < 1 || shape_order > 3) { set_error("hyb_pic_step: bad nsteps, np or shape_order"); return HYB_EINVAL; }
    if (np > 0 && (!cell || !off || !u || !qm || !q || !off_new || (p->g->d.dims == 2 && !v3))) {
        set_error("hyb_pic_step: null particle array (v3 is required in 2D)");
        return HYB_EINVAL;
    }
    if (!p->g->bound) { set_error("hyb_pic_step: fields not bound"); return HYB_ESTATE; }
    hyb_grid* g = p->g;
    auto step = [&]() {
        return g->d.precision == 32
            ? pic_step<float>(p, cell, (float*)off, (float*)u, (const float*)qm, (const float*)q, (float*)off_new, (float*)v3, np, shape_order)
            : pic_step<double>(p, cell, (double*)off, (double*)u, (const double*)qm, (const double*)q, (double*)off_new, (double*)v3, np, shape_order);
    };
    // A step is some twenty small launches and copies, so a call of several steps runs the first
    // one as plain launches (it imports k1-resident state if stale) and replays the rest as one
    // captured graph.  Not when the grid's fused kernel exchanges halo rows under a fresh epoch
    // each launch (n1 = 4096), nor while the caller is capturing its own graph.
    cudaStreamCaptureStatus outer = cudaStreamCaptureStatusNone;
    HYB_CUDA_TRY(cudaStreamIsCapturing(g->stream, &outer));
    const bool graphs = nsteps >= kPicGraphMinSteps && !(g->path == 2 && !g->resident && fused_epoch_launches(g)) &&
                        !g->ev_start && outer == cudaStreamCaptureStatusNone;
    if (!graphs) {
        for (int s = 0; s < nsteps; s++) {
            hyb_status st = step();
            if (st != HYB_OK) return st;
        }
        return HYB_OK;
    }
    hyb_status st = step();
    if (st != HYB_OK) return st;
    const void* key[12] = {cell, off, u, qm, q, off_new, v3, g->E[0], g->E[1], g->E[2], g->B[0], g->J[0]};
    bool same = p->exec && np == p->key_np && shape_order == p->key_order && g->path == p->key_path && g->resident == p->key_res;
    for (int i = 0; i < 12 && same; i++) same = key[i] == p->key[i];
    if (!p->cs) {
        HYB_CUDA_TRY(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking));
        HYB_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
        HYB_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    }
    cudaStream_t orig = g->stream;
    HYB_CUDA_TRY(cudaEventRecord(p->ev_fork, orig));
    HYB_CUDA_TRY(cudaStreamWaitEvent(p->cs, p->ev_fork, 0));
    if (!same) {
        if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
        cudaGraph_t graph = nullptr;
        g->stream = p->cs;
        cudaError_t ce = cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeRelaxed);
        if (ce == cudaSuccess) {
            st = step();
            ce = cudaStreamEndCapture(p->cs, &graph);
        }
        g->stream = orig;
        if (p->shadow) p->shadow->stream = orig;    // the captured step pointed it at the private stream
        if (st == HYB_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st != HYB_OK || ce != cudaSuccess) {
            // the captured step did not run: the remaining steps as plain launches
            if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
            cudaGetLastError();
            for (int s = 1; s < nsteps; s++) {
                st = step();
                if (st != HYB_OK) return st;
            }
            return HYB_OK;
        }
        for (int i = 0; i < 12; i++) p->key[i] = key[i];
        p->key_np = np;
        p->key_order = shape_order;
        p->key_path = g->path;
        p->key_res = g->resident;
    }
    for (int s = 1; s < nsteps; s++) HYB_CUDA_TRY(cudaGraphLaunch(p->exec, p->cs));
    HYB_CUDA_TRY(cudaEventRecord(p->ev_join, p->cs));
    HYB_CUDA_TRY(cudaStreamWaitEvent(orig, p->ev_join, 0));
    return HYB_OK;
}

hyb_status hyb_pic_destroy(hyb_pic* p) {
    if (!p) return HYB_OK;
    if (p->cs) cudaStreamSynchronize(p->cs);
    if (p->shadow) {
        p->shadow->stream = nullptr;      // never the private stream destroyed below (the caller's grid may be gone)
        hyb_destroy_grid(p->shadow);
    }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->cs) cudaStreamDestroy(p->cs);
    if (p->scratch) cudaFree(p->scratch);
    delete p;
    return HYB_OK;
}

}  // extern "C"
