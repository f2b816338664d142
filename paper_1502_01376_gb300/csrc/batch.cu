// batch.cu -- many independent grids advanced together, one CUDA-graph launch
// per step.  Grids that run the fused FP32 kernel are grouped by n1; each
// group is one persistent launch of k_fused_tmt (k_fused_tm for n1 = 4096)
// over a table of work items (grid, strip, first row, end row) from all its
// grids, after one launch that copies the halo rows of every group's items.
// Quasi-3D modes with nz = 2048 and a common radial grid are advanced together
// (z transform of all their arrays, leapfrog of all modes, inverse: three
// launches for up to eight modes).  Other grids (FP64, 3D, unsupported n1, other
// quasi-3D modes) run their own step.
// Groups, and each of the other grids, are forked onto side streams inside the
// captured graph so that they overlap.  hyb_batch_tune times candidate strip heights per group on scratch
// fields and keeps the fastest (the autotuner).
#include <algorithm>
#include <vector>

#include "fused_api.cuh"

struct hyb_batch {
    std::vector<hyb_grid*> grids;
    cudaStream_t stream = nullptr;
    struct Group {
        int n1 = 0;
        std::vector<int> members;          // indices into grids
        int rows_per_strip = 8;            // tuned
        int4* items = nullptr;             // device work items
        int n_items = 0;
        int grid = 0;
        std::vector<int4> h_items;         // host copy of the work items
        cudaStream_t side = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
    };
    std::vector<Group> groups;
    std::vector<int> q3;                   // quasi-3D modes advanced together (quasi3d_advance_many)
    cudaStream_t q3side = nullptr;
    cudaEvent_t q3fork = nullptr, q3join = nullptr;
    std::vector<int> others;               // other grids (three-pass path, other quasi-3D modes)
    std::vector<cudaStream_t> oside;       // one side stream (and fork/join events) per other grid
    std::vector<cudaEvent_t> ofork, ojoin;
    hyb::RowCopy* halo_tasks = nullptr;    // device: the halo rows of all groups' items
    int n_halo = 0, halo_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    int launches_per_step = 0;
};

namespace hyb {

static hyb_status group_plan(hyb_batch* b, hyb_batch::Group& G) {
    std::vector<int4> items;
    for (size_t k = 0; k < G.members.size(); k++) {
        hyb_grid* g = b->grids[G.members[k]];
        int ns = (g->d.n2 + G.rows_per_strip - 1) / G.rows_per_strip;
        if (ns > g->d.n2 / 2) ns = g->d.n2 / 2;
        if (ns < 1) ns = 1;
        hyb_status st = fused_set_strips(g, ns);
        if (st != HYB_OK) return st;
        std::vector<int4> it = fused_items((int)k, g->d.n2, ns);
        items.insert(items.end(), it.begin(), it.end());
    }
    // longest items first, so that the persistent CTAs finish together
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& c) { return (a.w - a.z) > (c.w - c.z); });
    if (G.items) { cudaFree(G.items); G.items = nullptr; }
    HYB_CUDA_TRY(cudaMalloc(&G.items, sizeof(int4) * items.size()));
    HYB_CUDA_TRY(cudaMemcpy(G.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    G.n_items = (int)items.size();
    G.h_items = items;
    int occ = 0, sms = 0;
    HYB_CUDA_TRY(fused_occupancy(G.n1, &occ));
    HYB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->grids[0]->device));
    G.grid = std::min(G.n_items, sms * occ);
    b->dirty = true;
    return HYB_OK;
}

static FusedBatch group_args(hyb_batch* b, const hyb_batch::Group& G) {
    FusedBatch fb;
    for (size_t k = 0; k < G.members.size(); k++) fb.inst[k] = fused_inst(b->grids[G.members[k]]);
    fb.items = G.items;
    fb.n_items = G.n_items;
    fb.flags = nullptr;                  // halo-buffer mode (work items may outnumber CTAs)
    fb.epoch = 0;
    fb.n_strips = 0;
    fb.err = b->grids[G.members[0]]->dflag;   // a device wait that gives up is reported by hyb_check of this grid
    return fb;
}

// the halo rows of every group's work items (E1, E2, E3, B1, B3 of row p0 - 1; E1, E3 of row p1),
// from the bound arrays into each grid's halo buffer: the task table of the one copy launch
static hyb_status halo_plan(hyb_batch* b) {
    std::vector<RowCopy> tasks;
    for (auto& G : b->groups) {
        for (const int4& it : G.h_items) {
            const hyb_grid* g = b->grids[G.members[it.x]];
            const FusedInst a = fused_inst(g);
            const int n1 = G.n1, n2 = a.n2, rl = (it.z - 1 + n2) % n2, rn = it.w % n2;
            const float* src[7] = {a.E[0] + (size_t)rl * n1, a.E[1] + (size_t)rl * n1, a.E[2] + (size_t)rl * n1,
                                   a.B[0] + (size_t)rl * n1, a.B[2] + (size_t)rl * n1, a.E[0] + (size_t)rn * n1,
                                   a.E[2] + (size_t)rn * n1};
            for (int k = 0; k < 7; k++)
                tasks.push_back(RowCopy{src[k], const_cast<float*>(a.halo) + ((size_t)it.y * 7 + k) * n1, n1, 0});
        }
    }
    if ((int)tasks.size() > b->halo_cap) {
        if (b->halo_tasks) cudaFree(b->halo_tasks);
        b->halo_tasks = nullptr;
        b->halo_cap = 0;
        HYB_CUDA_TRY(cudaMalloc(&b->halo_tasks, sizeof(RowCopy) * tasks.size()));
        b->halo_cap = (int)tasks.size();
    }
    if (!tasks.empty())
        HYB_CUDA_TRY(cudaMemcpy(b->halo_tasks, tasks.data(), sizeof(RowCopy) * tasks.size(), cudaMemcpyHostToDevice));
    b->n_halo = (int)tasks.size();
    return HYB_OK;
}

// enqueue one step: the others forked onto side streams, the halo copy of all groups, then
// every group (forked onto side streams)
static hyb_status enqueue_step(hyb_batch* b, cudaStream_t s) {
    if (!b->q3.empty()) {
        std::vector<hyb_grid*> gs;
        for (int i : b->q3) gs.push_back(b->grids[i]);
        HYB_CUDA_TRY(cudaEventRecord(b->q3fork, s));
        HYB_CUDA_TRY(cudaStreamWaitEvent(b->q3side, b->q3fork, 0));
        hyb_status st = quasi3d_advance_many(gs.data(), (int)gs.size(), b->q3side);
        if (st != HYB_OK) return st;
        HYB_CUDA_TRY(cudaEventRecord(b->q3join, b->q3side));
    }
    for (size_t o = 0; o < b->others.size(); o++) {
        hyb_grid* g = b->grids[b->others[o]];
        HYB_CUDA_TRY(cudaEventRecord(b->ofork[o], s));
        HYB_CUDA_TRY(cudaStreamWaitEvent(b->oside[o], b->ofork[o], 0));
        cudaStream_t keep = g->stream;
        g->stream = b->oside[o];
        hyb_status st = g->d.dims == 20 ? quasi3d_advance(g, 1)
                       : g->d.precision == 32 ? generic_advance<float>(g, 1) : generic_advance<double>(g, 1);
        g->stream = keep;
        if (st != HYB_OK) return st;
        HYB_CUDA_TRY(cudaEventRecord(b->ojoin[o], b->oside[o]));
    }
    HYB_CUDA_TRY(copy_rows(b->halo_tasks, b->n_halo, s));
    for (auto& G : b->groups) {
        HYB_CUDA_TRY(cudaEventRecord(G.fork, s));
        HYB_CUDA_TRY(cudaStreamWaitEvent(G.side, G.fork, 0));
        HYB_CUDA_TRY(fused_kernel_launch(G.n1, group_args(b, G), G.grid, G.side));
        HYB_CUDA_TRY(cudaEventRecord(G.join, G.side));
    }
    for (auto& G : b->groups) HYB_CUDA_TRY(cudaStreamWaitEvent(s, G.join, 0));
    for (cudaEvent_t e : b->ojoin) HYB_CUDA_TRY(cudaStreamWaitEvent(s, e, 0));
    if (!b->q3.empty()) HYB_CUDA_TRY(cudaStreamWaitEvent(s, b->q3join, 0));
    return HYB_OK;
}

static hyb_status capture(hyb_batch* b) {
    hyb_status hs = halo_plan(b);
    if (hs != HYB_OK) return hs;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaStream_t cs = nullptr;
    HYB_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    HYB_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    hyb_status st = enqueue_step(b, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st != HYB_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = graph;
    HYB_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
    b->dirty = false;
    return HYB_OK;
}

}  // namespace hyb

using namespace hyb;

extern "C" {

hyb_status hyb_batch_create(const hyb_grid_desc* descs, int n, void* stream, hyb_batch** out) {
    if (!descs || !out || n < 1) { set_error("hyb_batch_create: bad arguments"); return HYB_EINVAL; }
    *out = nullptr;
    hyb_batch* b = new hyb_batch();
    b->stream = (cudaStream_t)stream;
    for (int i = 0; i < n; i++) {
        hyb_grid* g = nullptr;
        hyb_status st = hyb_create_grid(&descs[i], stream, &g);
        if (st != HYB_OK) { hyb_batch_destroy(b); return st; }
        b->grids.push_back(g);
    }
    for (int i = 0; i < n; i++) {
        hyb_grid* g = b->grids[i];
        if (g->d.dims == 20 && (b->q3.empty() ? quasi3d_can_batch(g, g) : quasi3d_can_batch(b->grids[b->q3[0]], g))) {
            b->q3.push_back(i);
            continue;
        }
        if (g->path != 2) { b->others.push_back(i); continue; }
        auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const hyb_batch::Group& G) { return G.n1 == g->d.n1; });
        if (it == b->groups.end()) {
            b->groups.emplace_back();
            b->groups.back().n1 = g->d.n1;
            it = b->groups.end() - 1;
        }
        if ((int)it->members.size() >= kMaxInst) { set_error("more than %d fused grids with the same n1", kMaxInst); hyb_batch_destroy(b); return HYB_EINVAL; }
        it->members.push_back(i);
    }
    for (auto& G : b->groups) {
        cudaError_t e = cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G.join, cudaEventDisableTiming);
        if (e != cudaSuccess) { hyb_status st = cuda_fail(e, "stream/event creation"); hyb_batch_destroy(b); return st; }
        hyb_status st = group_plan(b, G);
        if (st != HYB_OK) { hyb_batch_destroy(b); return st; }
    }
    if (!b->q3.empty()) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->q3side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->q3fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->q3join, cudaEventDisableTiming);
        if (e != cudaSuccess) { hyb_status st = cuda_fail(e, "stream/event creation"); hyb_batch_destroy(b); return st; }
    }
    for (size_t o = 0; o < b->others.size(); o++) {
        cudaStream_t st_ = nullptr;
        cudaEvent_t f = nullptr, j = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        b->oside.push_back(st_);
        b->ofork.push_back(f);
        b->ojoin.push_back(j);
        if (e != cudaSuccess) { hyb_status st = cuda_fail(e, "stream/event creation"); hyb_batch_destroy(b); return st; }
    }
    b->launches_per_step = (int)b->groups.size() + (b->groups.empty() ? 0 : 1);
    if (!b->q3.empty()) b->launches_per_step += 3 * (((int)b->q3.size() + 7) / 8);
    for (int i : b->others) b->launches_per_step += hyb_launches_per_step(b->grids[i]);
    *out = b;
    return HYB_OK;
}

hyb_status hyb_batch_bind(hyb_batch* b, int i, void* const E[3], void* const B[3], void* const J[3]) {
    if (!b || i < 0 || i >= (int)b->grids.size()) { set_error("hyb_batch_bind: bad index"); return HYB_EINVAL; }
    hyb_status st = hyb_bind_fields(b->grids[i], E, B, J, nullptr);
    if (st == HYB_OK) b->dirty = true;
    return st;
}

hyb_status hyb_batch_advance(hyb_batch* b, int nsteps) {
    if (!b || nsteps < 0) { set_error("hyb_batch_advance: bad arguments"); return HYB_EINVAL; }
    for (auto* g : b->grids) if (!g->bound) { set_error("hyb_batch_advance: a grid is not bound"); return HYB_ESTATE; }
    if (b->dirty) { hyb_status st = capture(b); if (st != HYB_OK) return st; }
    for (int s = 0; s < nsteps; s++) HYB_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    return HYB_OK;
}

hyb_status hyb_batch_tune(hyb_batch* b, int trials) {
    if (!b) { set_error("null batch"); return HYB_EINVAL; }
    if (trials < 1) trials = 3;
    static const int cand[] = {2, 3, 4, 6, 8, 12, 16, 24, 32};
    cudaEvent_t e0, e1;
    HYB_CUDA_TRY(cudaEventCreate(&e0));
    HYB_CUDA_TRY(cudaEventCreate(&e1));
    // each timed launch starts with a cold L2, as a group does inside a step (a write larger than
    // the L2 between launches): a group small enough to stay in L2 would otherwise be tuned warm
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->grids[0]->device);
    const size_t flush_bytes = (size_t)std::max(l2, 1 << 20) * 3 / 2;
    void* flush = nullptr;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) { flush = nullptr; cudaGetLastError(); }
    hyb_status result = HYB_OK;
    for (auto& G : b->groups) {
        // scratch fields: timing does not depend on the values
        std::vector<void*> bufs;
        bool fail = false;
        for (int m : G.members) {
            hyb_grid* g = b->grids[m];
            void* p = nullptr;
            if (cudaMalloc(&p, (size_t)9 * g->cells * sizeof(float)) != cudaSuccess) { fail = true; break; }
            cudaMemset(p, 0, (size_t)9 * g->cells * sizeof(float));
            bufs.push_back(p);
        }
        if (fail) { for (void* p : bufs) cudaFree(p); result = cuda_fail(cudaErrorMemoryAllocation, "hyb_batch_tune scratch"); break; }
        float best = 1e30f;
        int best_h = G.rows_per_strip;
        // candidates: a fixed ladder plus, for 1 to 3 waves of resident CTAs, the smallest
        // strip height whose work items fill that many waves
        std::vector<int> hs(cand, cand + sizeof(cand) / sizeof(cand[0]));
        {
            int occ = 1, sms = 1;
            if (fused_occupancy(G.n1, &occ) != cudaSuccess || occ < 1) occ = 1;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->grids[0]->device) != cudaSuccess) sms = 1;
            for (int w = 1; w <= 3; w++)
                for (int h = 2; h <= 64; h++) {
                    int64_t items = 0;
                    for (int m : G.members) items += (b->grids[m]->d.n2 + h - 1) / h;
                    if (items <= (int64_t)w * sms * occ) { hs.push_back(h); break; }
                }
            std::sort(hs.begin(), hs.end());
            hs.erase(std::unique(hs.begin(), hs.end()), hs.end());
        }
        for (int h : hs) {
            G.rows_per_strip = h;
            hyb_status st = group_plan(b, G);
            if (st != HYB_OK) { result = st; break; }
            FusedBatch fb;
            for (size_t k = 0; k < G.members.size(); k++) {
                hyb_grid* g = b->grids[G.members[k]];
                FusedInst a = fused_inst(g);
                float* base = (float*)bufs[k];
                for (int c = 0; c < 3; c++) {
                    a.E[c] = base + (size_t)c * g->cells;
                    a.B[c] = base + (size_t)(3 + c) * g->cells;
                    a.J[c] = base + (size_t)(6 + c) * g->cells;
                }
                fb.inst[k] = a;
            }
            fb.items = G.items;
            fb.n_items = G.n_items;
            fb.flags = nullptr;
            fb.epoch = 0;
            fb.n_strips = 0;
            fb.err = b->grids[G.members[0]]->dflag;
            fused_launch(G.n1, fb, G.grid, b->stream, nullptr, nullptr);       // warm
            float ms = 0.f;
            cudaError_t e = cudaSuccess;
            for (int t = 0; t < trials && e == cudaSuccess; t++) {
                if (flush) cudaMemsetAsync(flush, t & 0xff, flush_bytes, b->stream);
                cudaEventRecord(e0, b->stream);
                fused_launch(G.n1, fb, G.grid, b->stream, nullptr, nullptr);
                cudaEventRecord(e1, b->stream);
                e = cudaEventSynchronize(e1);
                float one = 0.f;
                if (e == cudaSuccess) cudaEventElapsedTime(&one, e0, e1);
                ms += one;
            }
            if (e != cudaSuccess) { result = cuda_fail(e, "hyb_batch_tune"); break; }
            if (ms < best) { best = ms; best_h = h; }
        }
        for (void* p : bufs) cudaFree(p);
        if (result != HYB_OK) break;
        G.rows_per_strip = best_h;
        result = group_plan(b, G);
        if (result != HYB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    b->dirty = true;
    return result;
}

int hyb_batch_rows_per_strip(const hyb_batch* b, int n1) {
    if (!b) return 0;
    for (auto& G : b->groups) if (G.n1 == n1) return G.rows_per_strip;
    return 0;
}

hyb_status hyb_batch_set_rows_per_strip(hyb_batch* b, int n1, int h) {
    if (!b) { set_error("null batch"); return HYB_EINVAL; }
    if (h < 1) { set_error("rows per strip must be >= 1"); return HYB_EINVAL; }
    for (auto& G : b->groups)
        if (G.n1 == n1) {
            G.rows_per_strip = h;
            return group_plan(b, G);
        }
    set_error("no fused group with this n1");
    return HYB_EINVAL;
}

int hyb_batch_launches_per_step(const hyb_batch* b) { return b ? b->launches_per_step : 0; }

hyb_status hyb_batch_destroy(hyb_batch* b) {
    if (!b) return HYB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->halo_tasks) cudaFree(b->halo_tasks);
    if (b->q3side) cudaStreamDestroy(b->q3side);
    if (b->q3fork) cudaEventDestroy(b->q3fork);
    if (b->q3join) cudaEventDestroy(b->q3join);
    for (auto& G : b->groups) {
        if (G.items) cudaFree(G.items);
        if (G.side) cudaStreamDestroy(G.side);
        if (G.fork) cudaEventDestroy(G.fork);
        if (G.join) cudaEventDestroy(G.join);
    }
    for (size_t o = 0; o < b->oside.size(); o++) {
        if (b->oside[o]) cudaStreamDestroy(b->oside[o]);
        if (b->ofork[o]) cudaEventDestroy(b->ofork[o]);
        if (b->ojoin[o]) cudaEventDestroy(b->ojoin[o]);
    }
    for (auto* g : b->grids) hyb_destroy_grid(g);
    delete b;
    return HYB_OK;
}

}  // extern "C"
