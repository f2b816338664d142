// batch.cu -- many independent grids advanced together, one CUDA-graph launch
// per step.  Grids that run the fused FP32 kernel are grouped by n1 and cut into
// work items (grid, strip, first row, end row); quasi-3D modes with nz = 2048 and
// a common radial grid are advanced together.  A step is either
//   * one persistent launch (batch_step.cu) whose CTAs are split into one role per
//     n1 group and one for the quasi-3D modes, when every grid belongs to one of
//     them; or
//   * a graph of launches: one copy of the halo rows of every group's items, one
//     persistent launch of k_fused_tmt (k_fused_tm for n1 = 4096) per group, three
//     launches for up to eight quasi-3D modes, and the own step of every other grid
//     (FP64, 3D, unsupported n1, other quasi-3D modes), forked onto side streams so
//     that they overlap.
// hyb_batch_tune (the autotuner) times candidate strip heights per group on scratch
// fields, then the split of the single launch's CTAs among its roles, and keeps the
// faster of the two forms of the step.
#include <algorithm>
#include <string>
#include <vector>

#include "batch_step.cuh"
#include "fused_api.cuh"

struct hyb_batch {
    std::vector<hyb_grid*> grids;
    cudaStream_t stream = nullptr;
    struct Group {
        int n1 = 0;
        std::vector<int> members;          // indices into grids
        int rows_per_strip = 8;            // tuned (graph of launches)
        int rows_single = 0;               // tuned for the single launch (0: rows_per_strip)
        int planned = 0;                   // the height the current work items were cut with
        int4* items = nullptr;             // device work items
        int n_items = 0;
        int grid = 0;
        std::vector<int4> h_items;         // host copy of the work items
        int halo0 = 0, n_halo = 0;         // its halo rows in the task table
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
    // the step as one persistent launch (batch_step.cu)
    bool single_ok = false;                // every grid belongs to a role of the single launch
    bool single = false;                   // steps use it
    int step_ctas = 0;                     // CTAs of the launch
    int role_ctas[hyb::kRoles] = {};       // CTAs of each role (0: no such role)
    unsigned* d_sync = nullptr;            // role barriers
    unsigned long long* d_stamp = nullptr; // per-role start and end times (autotuner)
    double role_ms[hyb::kRoles] = {};      // each role's duration in the tuner's best single launch
};

namespace hyb {

// strips of a grid of n2 rows for strip height h (at least two rows a strip)
static int strips_of(int n2, int h) { return std::max(1, std::min((n2 + h - 1) / h, n2 / 2)); }

// the strip height of the group in the current form of the step
static int form_height(const hyb_batch* b, const hyb_batch::Group& G) {
    return b->single && G.rows_single > 0 ? G.rows_single : G.rows_per_strip;
}

// cuts the group's grids into work items of strip height h
static hyb_status group_plan(hyb_batch* b, hyb_batch::Group& G, int h) {
    std::vector<int4> items;
    for (size_t k = 0; k < G.members.size(); k++) {
        hyb_grid* g = b->grids[G.members[k]];
        const int ns = strips_of(g->d.n2, h);
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
    G.planned = h;
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
        G.halo0 = (int)tasks.size();
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
        G.n_halo = (int)tasks.size() - G.halo0;
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

// the arguments of the single launch: roles in the order of kRoleTM .. kRoleQ3, each on the next
// role_ctas[r] CTAs
static StepArgs step_args(hyb_batch* b, unsigned long long* stamp) {
    StepArgs a{};
    int cta = 0;
    for (auto& G : b->groups) {
        const int r = role_of_n1(G.n1);
        a.r2[r].fb = group_args(b, G);
        a.r2[r].halo = b->halo_tasks + G.halo0;
        a.r2[r].n_halo = G.n_halo;
    }
    for (int r = 0; r < 4; r++) {
        a.r2[r].cta0 = cta;
        a.r2[r].ncta = b->role_ctas[r];
        cta += b->role_ctas[r];
    }
    if (!b->q3.empty()) {
        std::vector<hyb_grid*> gs;
        for (int i : b->q3) gs.push_back(b->grids[i]);
        quasi3d_step_args(gs.data(), (int)gs.size(), &a.q3);
        a.q3_err = gs[0]->dflag;
    }
    a.q3_cta0 = cta;
    a.q3_ncta = b->role_ctas[kRoleQ3];
    a.sync = b->d_sync;
    a.stamp = stamp;
    return a;
}

// CTAs per role in proportion to the work estimates w[r] (at least one CTA for a role with work)
static void split_ctas(hyb_batch* b, const double* w) {
    double tot = 0.0;
    for (int r = 0; r < kRoles; r++) if (w[r] > 0.0) tot += w[r];
    int used = 0, big = -1;
    for (int r = 0; r < kRoles; r++) {
        b->role_ctas[r] = 0;
        if (w[r] <= 0.0) continue;
        b->role_ctas[r] = std::max(1, (int)std::lround(b->step_ctas * w[r] / tot));
        used += b->role_ctas[r];
        if (big < 0 || b->role_ctas[r] > b->role_ctas[big]) big = r;
    }
    // the rounding error goes to the largest role; if the minimum of one CTA per role overshot,
    // take the excess from the largest roles
    if (big >= 0) b->role_ctas[big] += b->step_ctas - used;
    while (big >= 0 && b->role_ctas[big] < 1) {
        int donor = -1;
        for (int r = 0; r < kRoles; r++)
            if (r != big && b->role_ctas[r] > 1 && (donor < 0 || b->role_ctas[r] > b->role_ctas[donor])) donor = r;
        if (donor < 0) break;
        b->role_ctas[donor]--;
        b->role_ctas[big]++;
    }
}

// a first split (before hyb_batch_tune) from the bytes each role moves, 60 B per 2D cell and 360 B
// per quasi-3D point over the three stages, and the rate each role reached in the tuned single
// launch of a 16-grid + 3-mode batch, per CTA, scaled to 152 CTAs (TB/s)
static void default_split(hyb_batch* b) {
    double w[kRoles] = {0, 0, 0, 0, 0};
    static const double rate[4] = {2.6, 3.4, 2.9, 2.8};
    for (auto& G : b->groups) {
        int64_t cells = 0;
        for (int m : G.members) cells += b->grids[m]->cells;
        w[role_of_n1(G.n1)] += 60.0 * (double)cells / rate[role_of_n1(G.n1)];
    }
    for (int i : b->q3) w[kRoleQ3] += 360.0 * (double)b->grids[i]->cells / 6.2;
    split_ctas(b, w);
}

static void count_launches(hyb_batch* b) {
    if (b->single) { b->launches_per_step = 1; return; }
    b->launches_per_step = (int)b->groups.size() + (b->groups.empty() ? 0 : 1);
    if (!b->q3.empty()) b->launches_per_step += 3 * (((int)b->q3.size() + 7) / 8);
    for (int i : b->others) b->launches_per_step += hyb_launches_per_step(b->grids[i]);
}

// enqueue one step.  Single launch: the one persistent launch.  Otherwise the others forked onto
// side streams, the halo copy of all groups, then every group (forked onto side streams)
static hyb_status enqueue_step(hyb_batch* b, cudaStream_t s) {
    if (b->single) {
        HYB_CUDA_TRY(batch_step_launch(step_args(b, nullptr), b->step_ctas, s));
        return HYB_OK;
    }
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

// work items cut for the current form of the step, and their halo rows
static hyb_status plan(hyb_batch* b) {
    for (auto& G : b->groups)
        if (G.planned != form_height(b, G)) {
            hyb_status st = group_plan(b, G, form_height(b, G));
            if (st != HYB_OK) return st;
        }
    return halo_plan(b);
}

static hyb_status capture(hyb_batch* b) {
    hyb_status hs = plan(b);
    if (hs != HYB_OK) return hs;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (b->single) HYB_CUDA_TRY(cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned) * 2 * kRoles, b->stream));
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

// mean time of `trials` steps of the current form, each after a write larger than the L2
static hyb_status time_steps(hyb_batch* b, int trials, cudaEvent_t e0, cudaEvent_t e1, void* flush, size_t flush_bytes,
                             float* ms_out) {
    hyb_status st = capture(b);
    if (st != HYB_OK) return st;
    HYB_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));           // warm
    float ms = 0.f;
    for (int t = 0; t < trials; t++) {
        if (flush) HYB_CUDA_TRY(cudaMemsetAsync(flush, t & 0xff, flush_bytes, b->stream));
        HYB_CUDA_TRY(cudaEventRecord(e0, b->stream));
        HYB_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
        HYB_CUDA_TRY(cudaEventRecord(e1, b->stream));
        HYB_CUDA_TRY(cudaEventSynchronize(e1));
        float one = 0.f;
        HYB_CUDA_TRY(cudaEventElapsedTime(&one, e0, e1));
        ms += one;
    }
    *ms_out = ms / (float)trials;
    return HYB_OK;
}

// one single launch per trial, each after a write larger than the L2: the mean time and each
// role's mean duration (first CTA start to last CTA end)
static cudaError_t run_single(hyb_batch* b, int trials, cudaEvent_t e0, cudaEvent_t e1, void* flush, size_t flush_bytes,
                              float* ms_out, double* dur) {
    const StepArgs a = step_args(b, b->d_stamp);
    for (int r = 0; r < kRoles; r++) dur[r] = 0.0;
    cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned) * 2 * kRoles, b->stream);
    if (e == cudaSuccess) e = batch_step_launch(a, b->step_ctas, b->stream);          // warm
    float ms = 0.f;
    for (int t = 0; t < trials && e == cudaSuccess; t++) {
        unsigned long long init[2 * kRoles];
        for (int r = 0; r < kRoles; r++) { init[2 * r] = ~0ull; init[2 * r + 1] = 0ull; }
        e = cudaMemcpyAsync(b->d_stamp, init, sizeof(init), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess && flush) e = cudaMemsetAsync(flush, t & 0xff, flush_bytes, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = batch_step_launch(a, b->step_ctas, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float one = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&one, e0, e1);
        ms += one;
        unsigned long long st[2 * kRoles];
        if (e == cudaSuccess) e = cudaMemcpy(st, b->d_stamp, sizeof(st), cudaMemcpyDeviceToHost);
        for (int r = 0; r < kRoles && e == cudaSuccess; r++)
            if (b->role_ctas[r] > 0 && st[2 * r + 1] > st[2 * r]) dur[r] += 1e-6 * (double)(st[2 * r + 1] - st[2 * r]);
    }
    *ms_out = ms / (float)trials;
    for (int r = 0; r < kRoles; r++) dur[r] /= trials;
    return e;
}

// candidate strip heights of a group whose work items share `units` strip sweepers: a fixed
// ladder plus, for 1 to 4 waves of the sweepers, the smallest height whose items fit that many
static std::vector<int> single_candidates(const hyb_batch* b, const hyb_batch::Group& G, int units) {
    std::vector<int> hs = {2, 3, 4, 6, 8, 12, 16, 24, 32};
    for (int w = 1; w <= 4; w++)
        for (int h = 2; h <= 256; h++) {
            int64_t items = 0;
            for (int m : G.members) items += strips_of(b->grids[m]->d.n2, h);
            if (items <= (int64_t)w * units) { hs.push_back(h); break; }
        }
    std::sort(hs.begin(), hs.end());
    hs.erase(std::unique(hs.begin(), hs.end()), hs.end());
    return hs;
}

// cuts every group's work items with its single-launch height
static hyb_status plan_single(hyb_batch* b) {
    for (auto& G : b->groups) {
        hyb_status st = group_plan(b, G, G.rows_single);
        if (st != HYB_OK) return st;
    }
    return halo_plan(b);
}

// for the current split, each group of a role in `mask` takes the candidate strip height under
// which its role finished first (the groups' candidates timed together, in the same launches)
static hyb_status pick_heights(hyb_batch* b, unsigned mask, int trials, cudaEvent_t e0, cudaEvent_t e1, void* flush,
                               size_t flush_bytes) {
    static const int kTeams[4] = {1, 8, 4, 2};                   // strip sweepers per CTA of each 2D role
    const size_t ng = b->groups.size();
    std::vector<std::vector<int>> cand(ng);
    std::vector<double> dbest(ng, 1e30);
    std::vector<int> hbest(ng);
    size_t nc = 0;
    for (size_t k = 0; k < ng; k++) {
        const int r = role_of_n1(b->groups[k].n1);
        hbest[k] = b->groups[k].rows_single;
        if (!((mask >> r) & 1u)) continue;
        cand[k] = single_candidates(b, b->groups[k], kTeams[r] * b->role_ctas[r]);
        nc = std::max(nc, cand[k].size());
    }
    for (size_t c = 0; c < nc; c++) {
        for (size_t k = 0; k < ng; k++)
            if (!cand[k].empty()) b->groups[k].rows_single = cand[k][std::min(c, cand[k].size() - 1)];
        hyb_status st = plan_single(b);
        if (st != HYB_OK) return st;
        float ms = 0.f;
        double dur[kRoles];
        cudaError_t e = run_single(b, trials, e0, e1, flush, flush_bytes, &ms, dur);
        if (e != cudaSuccess) return cuda_fail(e, "hyb_batch_tune (single launch)");
        for (size_t k = 0; k < ng; k++) {
            const double d = dur[role_of_n1(b->groups[k].n1)];
            if (!cand[k].empty() && d < dbest[k]) { dbest[k] = d; hbest[k] = b->groups[k].rows_single; }
        }
    }
    for (size_t k = 0; k < ng; k++) b->groups[k].rows_single = hbest[k];
    return plan_single(b);
}

// the autotuner's second part, on the bound fields (saved first and restored at the end, so that
// tuning leaves them as they were).  (1) Rounds of: each group's strip height for the current split
// of the single launch's CTAs (pick_heights), then a new split with CTAs in proportion to each
// role's CTA time (CTAs x duration), until the split repeats.  (2) From the fastest of those, one
// CTA each to the roles that finished last (within 1 % of the last) from other roles (tried in the
// order of the duration they would have with one CTA less, in proportion; up to three choices),
// the changed roles' heights picked again, while the launch gets faster (the proportional split is
// coarse for roles of a few CTAs, whose durations also step with the waves of their work items).
// (3) The faster of the single launch and the graph of launches, each timed as its captured graph.
static hyb_status tune_single(hyb_batch* b, int trials, cudaEvent_t e0, cudaEvent_t e1, void* flush, size_t flush_bytes) {
    for (auto* g : b->grids) if (!g->bound) return HYB_OK;     // nothing to run on yet: keep the first split
    hyb_status hs = halo_plan(b);
    if (hs != HYB_OK) return hs;
    struct Saved { void* dst; void* copy; size_t bytes; };
    std::vector<Saved> saved;
    hyb_status result = HYB_OK;
    for (auto* g : b->grids) {
        const size_t bytes = (size_t)g->cells * (g->d.dims == 20 ? 2 : 1) * (size_t)(g->d.precision / 8);
        for (int c = 0; c < 6 && result == HYB_OK; c++) {
            void* dst = c < 3 ? g->E[c] : g->B[c - 3];
            void* copy = nullptr;
            cudaError_t e = cudaMalloc(&copy, bytes);
            if (e != cudaSuccess) { result = cuda_fail(e, "hyb_batch_tune copies"); break; }
            saved.push_back(Saved{dst, copy, bytes});
            e = cudaMemcpyAsync(copy, dst, bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) result = cuda_fail(e, "hyb_batch_tune copies");
        }
    }
    const bool keep_single = b->single;
    b->single = true;
    for (auto& G : b->groups) if (G.rows_single < 1) G.rows_single = G.rows_per_strip;
    float best = 1e30f;
    int best_split[kRoles];
    std::vector<int> best_h(b->groups.size());
    auto keep_best = [&](float ms, const double* dur) {
        best = ms;
        std::copy(b->role_ctas, b->role_ctas + kRoles, best_split);
        for (size_t k = 0; k < b->groups.size(); k++) best_h[k] = b->groups[k].rows_single;
        std::copy(dur, dur + kRoles, b->role_ms);
    };
    auto restore_best = [&]() {
        std::copy(best_split, best_split + kRoles, b->role_ctas);
        for (size_t k = 0; k < b->groups.size(); k++) b->groups[k].rows_single = best_h[k];
        return plan_single(b);
    };
    auto measure = [&](float* ms, double* dur) -> hyb_status {
        cudaError_t e = run_single(b, trials, e0, e1, flush, flush_bytes, ms, dur);
        return e == cudaSuccess ? HYB_OK : cuda_fail(e, "hyb_batch_tune (single launch)");
    };
    std::copy(b->role_ctas, b->role_ctas + kRoles, best_split);
    for (size_t k = 0; k < b->groups.size(); k++) best_h[k] = b->groups[k].rows_single;
    // (1)
    for (int iter = 0; iter < 6 && result == HYB_OK; iter++) {
        result = pick_heights(b, ~0u, trials, e0, e1, flush, flush_bytes);
        float ms = 0.f;
        double dur[kRoles];
        if (result == HYB_OK) result = measure(&ms, dur);
        if (result != HYB_OK) break;
        if (ms < best) keep_best(ms, dur);
        double w[kRoles];
        for (int r = 0; r < kRoles; r++) w[r] = b->role_ctas[r] > 0 ? (double)b->role_ctas[r] * std::max(dur[r], 1e-3) : 0.0;
        int prev[kRoles];
        std::copy(b->role_ctas, b->role_ctas + kRoles, prev);
        split_ctas(b, w);
        if (std::equal(prev, prev + kRoles, b->role_ctas)) break;
    }
    // (2)
    if (result == HYB_OK) result = restore_best();
    for (int iter = 0; iter < 16 && result == HYB_OK; iter++) {
        double dur[kRoles];
        std::copy(b->role_ms, b->role_ms + kRoles, dur);
        double top = 0.0;
        for (int r = 0; r < kRoles; r++) if (b->role_ctas[r] > 0) top = std::max(top, dur[r]);
        std::vector<int> slow;                                    // the roles that finish last
        std::vector<std::pair<double, int>> donors;               // the others, by their duration with one CTA less
        for (int r = 0; r < kRoles; r++) {
            if (b->role_ctas[r] < 1) continue;
            if (dur[r] >= 0.99 * top) slow.push_back(r);
            else if (b->role_ctas[r] > 1) donors.push_back({dur[r] * b->role_ctas[r] / (b->role_ctas[r] - 1), r});
        }
        std::sort(donors.begin(), donors.end());
        bool moved = false;
        // choice c: the slow roles take one CTA each from the donors c, c + 1, ... (a donor gives one)
        for (size_t c = 0; c < 3 && c + slow.size() <= donors.size() && !moved && result == HYB_OK; c++) {
            if (donors[c + slow.size() - 1].first >= top) break;
            result = restore_best();
            if (result != HYB_OK) break;
            unsigned mask = 0;
            for (size_t i = 0; i < slow.size(); i++) {
                const int from = donors[c + i].second;
                b->role_ctas[from]--;
                b->role_ctas[slow[i]]++;
                mask |= (1u << from) | (1u << slow[i]);
            }
            result = pick_heights(b, mask, trials, e0, e1, flush, flush_bytes);
            float ms = 0.f;
            double nd[kRoles];
            if (result == HYB_OK) result = measure(&ms, nd);
            if (result == HYB_OK && ms < best) { keep_best(ms, nd); moved = true; }
        }
        if (!moved) break;
    }
    if (result == HYB_OK) result = restore_best();
    // (3)
    b->single = keep_single;
    if (result == HYB_OK) {
        float t_single = 0.f, t_multi = 0.f;
        b->single = true;
        result = time_steps(b, trials, e0, e1, flush, flush_bytes, &t_single);
        if (result == HYB_OK) {
            b->single = false;
            result = time_steps(b, trials, e0, e1, flush, flush_bytes, &t_multi);
        }
        b->single = result == HYB_OK ? t_single <= t_multi : keep_single;
    }
    for (const Saved& sv : saved) {
        cudaError_t e = cudaMemcpyAsync(sv.dst, sv.copy, sv.bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess && result == HYB_OK) result = cuda_fail(e, "hyb_batch_tune restore");
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess && result == HYB_OK) result = cuda_fail(e, "hyb_batch_tune restore");
    for (const Saved& sv : saved) cudaFree(sv.copy);
    count_launches(b);
    b->dirty = true;
    return result;
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
        hyb_status st = group_plan(b, G, G.rows_per_strip);
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
    // the single launch: every grid in a role, at most one launch's worth of quasi-3D modes,
    // one CTA per SM for every role
    {
        bool ok = b->others.empty() && (int)b->q3.size() <= kQModes && !(b->groups.empty() && b->q3.empty());
        for (auto& G : b->groups) ok = ok && role_of_n1(G.n1) >= 0;
        if (ok && !b->q3.empty()) {
            std::vector<hyb_grid*> gs;
            for (int i : b->q3) gs.push_back(b->grids[i]);
            Q3Args qa;
            ok = quasi3d_step_args(gs.data(), (int)gs.size(), &qa) == HYB_OK;
        }
        int ctas = 0;
        int roles = (int)b->groups.size() + (b->q3.empty() ? 0 : 1);
        if (ok && (batch_step_ctas(&ctas) != cudaSuccess || ctas < roles)) { ok = false; cudaGetLastError(); }
        if (ok) {
            cudaError_t e = cudaMalloc(&b->d_sync, sizeof(unsigned) * 2 * kRoles);
            if (e == cudaSuccess) e = cudaMalloc(&b->d_stamp, sizeof(unsigned long long) * 2 * kRoles);
            if (e == cudaSuccess) e = cudaMemset(b->d_sync, 0, sizeof(unsigned) * 2 * kRoles);
            if (e != cudaSuccess) { hyb_status st = cuda_fail(e, "hyb_batch_create"); hyb_batch_destroy(b); return st; }
            b->step_ctas = ctas;
            default_split(b);
        }
        b->single_ok = ok;
        b->single = ok;
    }
    count_launches(b);
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
                    for (int m : G.members) items += strips_of(b->grids[m]->d.n2, h);
                    if (items <= (int64_t)w * sms * occ) { hs.push_back(h); break; }
                }
            std::sort(hs.begin(), hs.end());
            hs.erase(std::unique(hs.begin(), hs.end()), hs.end());
        }
        for (int h : hs) {
            G.rows_per_strip = h;
            hyb_status st = group_plan(b, G, h);
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
        result = group_plan(b, G, best_h);
        if (result != HYB_OK) break;
    }
    if (result == HYB_OK && b->single_ok) result = tune_single(b, trials, e0, e1, flush, flush_bytes);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFree(flush);
    b->dirty = true;
    return result;
}

int hyb_batch_rows_per_strip(const hyb_batch* b, int n1) {
    if (!b) return 0;
    for (auto& G : b->groups) if (G.n1 == n1) return form_height(b, G);
    return 0;
}

hyb_status hyb_batch_set_rows_per_strip(hyb_batch* b, int n1, int h) {
    if (!b) { set_error("null batch"); return HYB_EINVAL; }
    if (h < 1) { set_error("rows per strip must be >= 1"); return HYB_EINVAL; }
    for (auto& G : b->groups)
        if (G.n1 == n1) {
            G.rows_per_strip = G.rows_single = h;
            return group_plan(b, G, h);
        }
    set_error("no fused group with this n1");
    return HYB_EINVAL;
}

int hyb_batch_launches_per_step(const hyb_batch* b) { return b ? b->launches_per_step : 0; }

hyb_status hyb_batch_set_single_launch(hyb_batch* b, int on) {
    if (!b) { set_error("null batch"); return HYB_EINVAL; }
    if (on && !b->single_ok) { set_error("hyb_batch_set_single_launch: some grid has no role in the single launch"); return HYB_EINVAL; }
    b->single = on != 0;
    count_launches(b);
    b->dirty = true;
    return HYB_OK;
}

int hyb_batch_single_launch(const hyb_batch* b) { return b && b->single ? 1 : 0; }

hyb_status hyb_batch_check(hyb_batch* b) {
    if (!b) { set_error("null batch"); return HYB_EINVAL; }
    // every grid's flag is read and cleared; the first error found is the one reported
    hyb_status first = HYB_OK;
    std::string msg;
    for (auto* g : b->grids) {
        const hyb_status st = hyb_check(g);
        if (st != HYB_OK && first == HYB_OK) { first = st; msg = hyb_last_error(); }
    }
    if (first != HYB_OK) set_error("%s", msg.c_str());
    return first;
}

int hyb_batch_role_ctas(const hyb_batch* b, int role) {
    return b && role >= 0 && role < kRoles && b->single_ok ? b->role_ctas[role] : 0;
}

hyb_status hyb_batch_set_role_ctas(hyb_batch* b, const int* ctas) {
    if (!b || !ctas) { set_error("hyb_batch_set_role_ctas: null argument"); return HYB_EINVAL; }
    if (!b->single_ok) { set_error("hyb_batch_set_role_ctas: the batch has no single launch"); return HYB_EINVAL; }
    int sum = 0;
    for (int r = 0; r < kRoles; r++) {
        const bool present = b->role_ctas[r] > 0;
        if (present ? ctas[r] < 1 : ctas[r] != 0) {
            set_error("hyb_batch_set_role_ctas: role %d needs %s", r, present ? "at least one CTA" : "zero CTAs");
            return HYB_EINVAL;
        }
        sum += ctas[r];
    }
    if (sum > b->step_ctas) { set_error("hyb_batch_set_role_ctas: %d CTAs, more than the %d of the launch", sum, b->step_ctas); return HYB_EINVAL; }
    std::copy(ctas, ctas + kRoles, b->role_ctas);
    b->dirty = true;
    return HYB_OK;
}

double hyb_batch_role_ms(const hyb_batch* b, int role) {
    return b && role >= 0 && role < kRoles ? b->role_ms[role] : 0.0;
}

hyb_status hyb_batch_destroy(hyb_batch* b) {
    if (!b) return HYB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->halo_tasks) cudaFree(b->halo_tasks);
    if (b->d_sync) cudaFree(b->d_sync);
    if (b->d_stamp) cudaFree(b->d_stamp);
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
