// fused2d.cu -- host side of the single-pass FP32 hybrid advance for 2D grids
// (n1 = 512 .. 2048: k_fused_tmt of fused_tmt.cu; n1 = 4096: k_fused_tm of
// fused_tm.cu): the per-grid tables (per-mode symbols, twiddles), the strips of x2
// rows a grid is cut into (work items {instance, strip, p0, p1}), the halo rows
// (E1, E2, E3, B1, B3 of row p0 - 1 and E1, E3 of row p1, which neighbouring
// strips overwrite in place) copied by k_halo or k_copy_rows before a step unless
// the kernel exchanges them itself, the launch dispatch by n1, and the step from
// and to host arrays pipelined over chunks of rows.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fused_dev.cuh"

namespace hyb {

// copies the 7 halo rows of every work item: E1,E2,E3,B1,B3 of row p0-1 and E1,E3 of row p1
__global__ void k_halo(FusedBatch fb, int n1, int k0) {
    const int4 it = fb.items[blockIdx.x];
    const FusedInst& a = fb.inst[it.x];
    const int k = k0 + blockIdx.y;
    const int n2 = a.n2, p0 = it.z, p1 = it.w;
    const int rl = (p0 - 1 + n2) % n2, rn = p1 % n2;
    const float* src;
    switch (k) {
    case 0: src = a.E[0] + (size_t)rl * n1; break;
    case 1: src = a.E[1] + (size_t)rl * n1; break;
    case 2: src = a.E[2] + (size_t)rl * n1; break;
    case 3: src = a.B[0] + (size_t)rl * n1; break;
    case 4: src = a.B[2] + (size_t)rl * n1; break;
    case 5: src = a.E[0] + (size_t)rn * n1; break;
    default: src = a.E[2] + (size_t)rn * n1; break;
    }
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(const_cast<float*>(a.halo) + ((size_t)it.y * 7 + k) * n1);
    for (int i = threadIdx.x; i < n1 / 4; i += blockDim.x) d4[i] = s4[i];
}

// ------------------------------------------------------------------ host side
bool fused_supported(const hyb_grid_desc& d) {
    return d.precision == 32 && d.dims == 2 && (d.n1 == 512 || d.n1 == 1024 || d.n1 == 2048 || d.n1 == 4096) && d.n2 >= 4;
}

size_t fused_smem_bytes(int n1) { return n1 == 4096 ? fused_tm_smem_bytes() : fused_tmt_smem_bytes(n1); }

// work units (strips processed at once) per SM of the fused kernel for n1
cudaError_t fused_occupancy(int n1, int* occ) { return n1 == 4096 ? fused_tm_occupancy(occ) : fused_tmt_occupancy(n1, occ); }

// one step for the work items of a launch: halo copy (unless the kernel exchanges
// halos itself), then the persistent fused kernel
cudaError_t halo_parts(int n1, const FusedBatch& fb, int k0, int nk, cudaStream_t s) {
    if (fb.n_items < 1 || nk < 1) return cudaSuccess;
    k_halo<<<dim3(fb.n_items, nk), 256, 0, s>>>(fb, n1, k0);
    return cudaGetLastError();
}

// one warp per row task (rows are 2 to 16 KB), the tasks strided over a grid sized to the GPU, each
// lane four float4 in flight at a time
__global__ void k_copy_rows(const RowCopy* __restrict__ tasks, int n) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nw) copy_row_warp(tasks[w], lane);
}

cudaError_t copy_rows(const RowCopy* tasks, int n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    const int blocks = std::min((n + 7) / 8, resident_grid((const void*)k_copy_rows, 256, 0));
    k_copy_rows<<<blocks, 256, 0, s>>>(tasks, n);
    return cudaGetLastError();
}

cudaError_t fused_kernel_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s) {
    return n1 == 4096 ? fused_tm_launch(fb, grid, s) : fused_tmt_launch(n1, fb, grid, s);
}

cudaError_t fused_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e;
    if (!fb.flags) {
        e = halo_parts(n1, fb, 0, 7, s);
        if (e != cudaSuccess) return e;
    }
    if (ev0) { e = cudaEventRecord(ev0, s); if (e != cudaSuccess) return e; }
    e = fused_kernel_launch(n1, fb, grid, s);
    if (e != cudaSuccess) return e;
    if (ev1) e = cudaEventRecord(ev1, s);
    return e;
}

// per-grid tables of the fused kernel (symbols, W_N^c) and its halo buffer
hyb_status fused_tables(hyb_grid* g, int n_strips, FusedPlan* P) {
    const int N = g->d.n1, M = N / 2;
    std::vector<float2> S(M + 1);
    std::vector<float> cj1(M + 1), cj(M + 1);
    HYB_CUDA_TRY(cudaMemcpy(S.data(), g->tf.S, sizeof(float2) * (M + 1), cudaMemcpyDeviceToHost));
    HYB_CUDA_TRY(cudaMemcpy(cj1.data(), g->tf.cj1, sizeof(float) * (M + 1), cudaMemcpyDeviceToHost));
    HYB_CUDA_TRY(cudaMemcpy(cj.data(), g->tf.cj, sizeof(float) * (M + 1), cudaMemcpyDeviceToHost));
    std::vector<float4> sym(M + 1);
    for (int k = 0; k <= M; k++) sym[k] = make_float4(S[k].x, S[k].y, cj1[k], cj[k]);
    HYB_CUDA_TRY(cudaMalloc(&P->sym, sizeof(float4) * (M + 1)));
    HYB_CUDA_TRY(cudaMemcpy(P->sym, sym.data(), sizeof(float4) * (M + 1), cudaMemcpyHostToDevice));
    std::vector<float2> twC(256);
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < 256; c++) { const double ang = -2.0 * pi * c / N; twC[c] = make_float2((float)cos(ang), (float)sin(ang)); }
    HYB_CUDA_TRY(cudaMalloc(&P->twC, sizeof(float2) * 256));
    HYB_CUDA_TRY(cudaMemcpy(P->twC, twC.data(), sizeof(float2) * 256, cudaMemcpyHostToDevice));
    P->twM = g->tf.twM;
    HYB_CUDA_TRY(cudaMalloc(&P->halo, sizeof(float) * (size_t)n_strips * 7 * N));
    P->n_strips = n_strips;
    return HYB_OK;
}

// re-plans a fused grid for n_strips strips (halo buffer and single-grid items)
hyb_status fused_set_strips(hyb_grid* g, int n_strips) {
    FusedPlan* P = g->fused;
    if (n_strips < 1) n_strips = 1;
    if (n_strips > g->d.n2) n_strips = g->d.n2;
    if (P->halo) { cudaFree(P->halo); P->halo = nullptr; }
    HYB_CUDA_TRY(cudaMalloc(&P->halo, sizeof(float) * (size_t)n_strips * 7 * g->d.n1));
    P->n_strips = n_strips;
    std::vector<int4> it = fused_items(0, g->d.n2, n_strips);
    if (P->items) { cudaFree(P->items); P->items = nullptr; }
    HYB_CUDA_TRY(cudaMalloc(&P->items, sizeof(int4) * it.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    P->n_items = (int)it.size();
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(g->d.n1, &occ));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    P->grid = P->n_items < sms * occ ? P->n_items : sms * occ;
    if (P->flags) { cudaFree(P->flags); P->flags = nullptr; }
    if (P->n_items <= sms * occ && fused_in_kernel_halo(g->d.n1)) {
        HYB_CUDA_TRY(cudaMalloc(&P->flags, sizeof(int) * 2 * (size_t)n_strips));
        HYB_CUDA_TRY(cudaMemset(P->flags, 0, sizeof(int) * 2 * (size_t)n_strips));
        P->epoch = 0;
    }
    return HYB_OK;
}

// rows split into n_strips nearly equal strips: items {inst, strip, p0, p1}
std::vector<int4> fused_items(int inst, int n2, int n_strips) {
    std::vector<int4> it(n_strips);
    for (int s = 0; s < n_strips; s++)
        it[s] = make_int4(inst, s, (int)(((int64_t)s * n2) / n_strips), (int)(((int64_t)(s + 1) * n2) / n_strips));
    return it;
}

FusedInst fused_inst(const hyb_grid* g) {
    FusedInst a;
    const FusedPlan* P = g->fused;
    for (int c = 0; c < 3; c++) { a.E[c] = (float*)g->E[c]; a.B[c] = (float*)g->B[c]; a.J[c] = (const float*)g->J[c]; }
    a.halo = P->halo;
    a.sym = P->sym;
    a.twM = P->twM;
    a.twC = P->twC;
    a.a2 = (float)(g->d.dt / g->d.dx2);
    a.n2 = g->d.n2;
    return a;
}

// The halo rows of a single grid's strips are exchanged inside the kernel (one co-resident
// CTA per strip, cooperative launch) for n1 = 4096.  The n1 = 512 .. 2048 kernel runs two CTAs
// per SM, which the runtime's cooperative launch does not admit (it counts one per SM), so those
// grids copy their halo rows in a small launch before the step instead.
bool fused_in_kernel_halo(int n1) { return n1 == 4096; }

hyb_status fused_create(hyb_grid* g) {
    FusedPlan* P = new FusedPlan();
    g->fused = P;
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(g->d.n1, &occ));
    if (occ < 1) { set_error("fused kernel does not fit on an SM"); return HYB_EINVAL; }
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    int ns = sms * occ;
    if (ns > g->d.n2 / 2) ns = g->d.n2 / 2;
    if (ns < 1) ns = 1;
    hyb_status st = fused_tables(g, ns, P);
    if (st != HYB_OK) return st;
    std::vector<int4> it = fused_items(0, g->d.n2, ns);
    HYB_CUDA_TRY(cudaMalloc(&P->items, sizeof(int4) * it.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->items, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    P->n_items = (int)it.size();
    P->grid = (int)it.size();
    if (fused_in_kernel_halo(g->d.n1)) {
        HYB_CUDA_TRY(cudaMalloc(&P->flags, sizeof(int) * 2 * (size_t)ns));
        HYB_CUDA_TRY(cudaMemset(P->flags, 0, sizeof(int) * 2 * (size_t)ns));
    }
    P->epoch = 0;
    return HYB_OK;
}

static void hp_release(FusedPlan* P) {
    if (P->hp_items) cudaFree(P->hp_items);
    if (P->hp_halo) cudaFree(P->hp_halo);
    for (cudaStream_t& q : P->hp_s) { if (q) cudaStreamDestroy(q); q = nullptr; }
    for (cudaEvent_t e : P->hp_ev) if (e) cudaEventDestroy(e);
    P->hp_items = nullptr;
    P->hp_halo = nullptr;
    P->hp_ev.clear();
    P->hp_chunks = 0;
}

void fused_destroy(hyb_grid* g) {
    FusedPlan* P = g->fused;
    if (!P) return;
    hp_release(P);
    if (P->items) cudaFree(P->items);
    if (P->halo) cudaFree(P->halo);
    if (P->flags) cudaFree(P->flags);
    if (P->sym) cudaFree(P->sym);
    if (P->twC) cudaFree(P->twC);
    delete P;
    g->fused = nullptr;
}

hyb_status fused_advance(hyb_grid* g, int nsteps) {
    FusedPlan* P = g->fused;
    FusedBatch fb;
    fb.inst[0] = fused_inst(g);
    fb.items = P->items;
    fb.n_items = P->n_items;
    fb.flags = P->flags;          // in-kernel halo exchange: one co-resident CTA per strip
    fb.n_strips = P->n_strips;
    fb.err = g->dflag;
    for (int s = 0; s < nsteps; s++) {
        fb.epoch = ++P->epoch;
        HYB_CUDA_TRY(fused_launch(g->d.n1, fb, P->grid, g->stream, g->ev_start, g->ev_stop));
    }
    return HYB_OK;
}

int fused_launches_per_step(const hyb_grid* g) { return (g->fused && g->fused->flags) ? 1 : 2; }

// the grid's fused kernel exchanges halo rows in the kernel under a per-launch epoch
bool fused_epoch_launches(const hyb_grid* g) { return g->fused && g->fused->flags; }

const char* fused_step_kernel(const hyb_grid* g) {
    switch (g->d.n1) {
    case 512: return "k_fused_tmt<32>";
    case 1024: return "k_fused_tmt<64>";
    case 2048: return "k_fused_tmt<128>";
    default: return "k_fused_tm";
    }
}

// ------------------------------------------------------------------ one step from and to host arrays
// The copies over the host link dominate this step, so it is pipelined over chunks of rows:
// stream 0 copies the rows in (the last row first, then chunk by chunk), stream 1 fills the
// halo buffer and runs the fused kernel on chunk c as soon as chunks c and c + 1 have landed,
// stream 2 copies chunk c's E and B back once it is computed, while later chunks still come in.
// Halo rows must be taken before the rows they come from are updated in place: the lower
// parts of chunk c + 1 (row p0 - 1 of its strips, the first of which is the last row of chunk
// c) before chunk c runs, and the upper part of the very last strip (row 0) before chunk 0 runs.
static hyb_status hp_plan(hyb_grid* g) {
    FusedPlan* P = g->fused;
    if (P->hp_chunks) return HYB_OK;
    hp_release(P);                                 // whatever an earlier, failed plan left
    const int n2 = g->d.n2;
    const int C = std::max(1, std::min(4, n2 / 8));
    std::vector<int4> items;
    P->hp_first.assign(1, 0);
    P->hp_row0.assign(1, 0);
    for (int c = 0; c < C; c++) {
        const int r0 = (int)((int64_t)c * n2 / C), r1 = (int)((int64_t)(c + 1) * n2 / C);
        const int ns = std::max(1, (r1 - r0) / 2);
        for (int s = 0; s < ns; s++) {
            const int p0 = r0 + (int)((int64_t)s * (r1 - r0) / ns), p1 = r0 + (int)((int64_t)(s + 1) * (r1 - r0) / ns);
            items.push_back(make_int4(0, (int)items.size(), p0, p1));
        }
        P->hp_first.push_back((int)items.size());
        P->hp_row0.push_back(r1);
    }
    HYB_CUDA_TRY(cudaMalloc(&P->hp_items, sizeof(int4) * items.size()));
    HYB_CUDA_TRY(cudaMemcpy(P->hp_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    HYB_CUDA_TRY(cudaMalloc(&P->hp_halo, sizeof(float) * items.size() * 7 * (size_t)g->d.n1));
    for (auto& q : P->hp_s) HYB_CUDA_TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    P->hp_ev.assign(2 + 2 * (size_t)C, nullptr);
    for (auto& e : P->hp_ev) HYB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    P->hp_chunks = C;
    return HYB_OK;
}

hyb_status fused_host_advance(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3]) {
    hyb_status st = hp_plan(g);
    if (st != HYB_OK) return st;
    FusedPlan* P = g->fused;
    const int n1 = g->d.n1, n2 = g->d.n2, C = P->hp_chunks;
    const size_t rowb = sizeof(float) * (size_t)n1;
    cudaStream_t in = P->hp_s[0], cmp = P->hp_s[1], out = P->hp_s[2];
    cudaEvent_t fork = P->hp_ev[0], join = P->hp_ev[1];
    auto ev_in = [&](int c) { return P->hp_ev[2 + c]; };
    auto ev_cmp = [&](int c) { return P->hp_ev[2 + C + c]; };
    void* const* hf[3] = {E, B, J};
    void* df[3][3];
    for (int c = 0; c < 3; c++) { df[0][c] = g->E[c]; df[1][c] = g->B[c]; df[2][c] = g->J[c]; }
    auto rows_copy = [&](int kind, int comp, int r0, int r1, cudaMemcpyKind dir, cudaStream_t s) {
        char* d = (char*)df[kind][comp] + (size_t)r0 * rowb;
        char* h = (char*)hf[kind][comp] + (size_t)r0 * rowb;
        return dir == cudaMemcpyHostToDevice ? cudaMemcpyAsync(d, h, (size_t)(r1 - r0) * rowb, dir, s)
                                             : cudaMemcpyAsync(h, d, (size_t)(r1 - r0) * rowb, dir, s);
    };
    FusedBatch fb;
    fb.inst[0] = fused_inst(g);
    fb.inst[0].halo = P->hp_halo;
    fb.flags = nullptr;
    fb.epoch = 0;
    fb.n_strips = 0;
    fb.err = g->dflag;
    auto sub = [&](int i0, int i1) {
        FusedBatch b = fb;
        b.items = P->hp_items + i0;
        b.n_items = i1 - i0;
        return b;
    };
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(n1, &occ));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    const int last = P->hp_first[C] - 1;                   // the strip that ends at row n2 (wraps to row 0)
    // chunk ch's rows of all nine arrays, plus the first row of chunk ch + 1 for E1 and E3 (the
    // upper halo of the chunk's last strip), so that compute ch waits for its own copy only
    auto copy_in = [&](int ch) -> cudaError_t {
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) {
                const int extra = (k == 0 && c != 1 && ch + 1 < C) ? 1 : 0;
                cudaError_t e = rows_copy(k, c, P->hp_row0[ch], P->hp_row0[ch + 1] + extra, cudaMemcpyHostToDevice, in);
                if (e != cudaSuccess) return e;
            }
        return cudaEventRecord(ev_in(ch), in);
    };
    HYB_CUDA_TRY(cudaEventRecord(fork, g->stream));
    for (cudaStream_t q : P->hp_s) HYB_CUDA_TRY(cudaStreamWaitEvent(q, fork, 0));
    // the copy-in stream runs ahead chunk by chunk; compute ch waits for copy ch, copy-out ch for compute ch.
    // Halo rows are taken into the halo buffer before the chunk that holds them is updated.
    for (int k = 0; k < 3; k++)
        for (int c = 0; c < 3; c++) HYB_CUDA_TRY(rows_copy(k, c, n2 - 1, n2, cudaMemcpyHostToDevice, in));
    HYB_CUDA_TRY(copy_in(0));
    HYB_CUDA_TRY(cudaStreamWaitEvent(cmp, ev_in(0), 0));
    HYB_CUDA_TRY(halo_parts(n1, sub(last, last + 1), 5, 2, cmp));          // row 0, before chunk 0 runs
    HYB_CUDA_TRY(halo_parts(n1, sub(P->hp_first[0], P->hp_first[1]), 0, 5, cmp));
    for (int ch = 0; ch < C; ch++) {
        if (ch + 1 < C) HYB_CUDA_TRY(copy_in(ch + 1));
        const int i0 = P->hp_first[ch], i1 = P->hp_first[ch + 1];
        if (ch > 0) {
            HYB_CUDA_TRY(cudaStreamWaitEvent(cmp, ev_in(ch), 0));
            HYB_CUDA_TRY(halo_parts(n1, sub(i0 + 1, i1), 0, 5, cmp));      // lower halos inside chunk ch
        }
        HYB_CUDA_TRY(halo_parts(n1, sub(i0, ch + 1 == C ? i1 - 1 : i1), 5, 2, cmp));
        if (ch + 1 < C) HYB_CUDA_TRY(halo_parts(n1, sub(i1, i1 + 1), 0, 5, cmp));   // row r1 - 1, for chunk ch + 1
        const FusedBatch b = sub(i0, i1);
        HYB_CUDA_TRY(fused_kernel_launch(n1, b, std::min(b.n_items, sms * occ), cmp));
        HYB_CUDA_TRY(cudaEventRecord(ev_cmp(ch), cmp));
        HYB_CUDA_TRY(cudaStreamWaitEvent(out, ev_cmp(ch), 0));
        for (int k = 0; k < 2; k++)
            for (int c = 0; c < 3; c++) HYB_CUDA_TRY(rows_copy(k, c, P->hp_row0[ch], P->hp_row0[ch + 1], cudaMemcpyDeviceToHost, out));
    }
    HYB_CUDA_TRY(cudaEventRecord(join, out));
    HYB_CUDA_TRY(cudaStreamWaitEvent(g->stream, join, 0));
    return HYB_OK;
}

}  // namespace hyb
