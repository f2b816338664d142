// fused_api.cuh -- host-side interface of the fused FP32 2D kernel shared by
// the single-grid path (fused2d.cu) and the batched launch (batch.cu).
#pragma once
#include <vector>

#include "hyb_internal.cuh"

namespace hyb {

struct FusedInst {
    float* E[3];
    float* B[3];
    const float* J[3];
    const float* halo;   // [strips][7][n1] of this instance
    const float4* sym;   // per-mode {Re S, Im S, cj1, cj}
    const float2* twM;
    const float2* twC;
    float a2;            // c dt / dx2
    int n2;
};
constexpr int kMaxInst = 24;
struct FusedBatch {
    FusedInst inst[kMaxInst];
    const int4* items;   // {instance, strip, p0, p1}
    int n_items;
    // single-grid mode with in-kernel halo exchange (flags != nullptr): one
    // work item per CTA, all CTAs co-resident; halo[s] holds E1, E3 of strip
    // s's first row, published with flags[2 s] = epoch; flags[2 s + 1] = epoch
    // says strip s has read the row before it.
    int* flags;
    int epoch;
    int n_strips;
    int* err;
};

struct FusedPlan {
    int n_strips = 0;
    int4* items = nullptr;        // [n_items] {instance 0, strip, p0, p1} (device)
    int n_items = 0;
    int grid = 0;                 // CTAs of the persistent launch
    float* halo = nullptr;        // [n_strips][7][n1]
    int* flags = nullptr;         // [2 n_strips] in-kernel halo exchange
    int epoch = 0;
    float4* sym = nullptr;        // [M + 1] {Re S, Im S, cj1, cj}, S = c dt sigma+
    float2* twM = nullptr;        // [M] W_M^j (the grid's FP32 table)
    float2* twC = nullptr;        // [256] W_N^c
    // host-array step (fused_host_advance): the rows in chunks, each chunk in short strips,
    // with their own halo buffer, work items and three streams (copy in, compute, copy out)
    int hp_chunks = 0;
    int4* hp_items = nullptr;     // strips of all chunks in row order {0, strip, p0, p1}
    std::vector<int> hp_first;    // first item of chunk c (hp_chunks + 1 entries)
    std::vector<int> hp_row0;     // first row of chunk c (hp_chunks + 1 entries)
    float* hp_halo = nullptr;     // [strips][7][n1]
    cudaStream_t hp_s[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> hp_ev;   // fork, join, then per chunk: input landed, chunk computed
};

size_t fused_smem_bytes(int n1);
// n1 = 4096: the TMEM/TMA kernel (fused_tm.cu)
size_t fused_tm_smem_bytes();
cudaError_t fused_tm_occupancy(int* occ);
cudaError_t fused_tm_launch(const FusedBatch& fb, int grid, cudaStream_t s);
// n1 = 512, 1024, 2048 (fused_tmt.cu): occupancy and launches count work units (teams), not CTAs
size_t fused_tmt_smem_bytes(int n1);
cudaError_t fused_tmt_occupancy(int n1, int* units);
cudaError_t fused_tmt_launch(int n1, const FusedBatch& fb, int units, cudaStream_t s);
cudaError_t wait_probe(int* dflag, int* derr, long long limit, int which, cudaStream_t s);
cudaError_t fused_occupancy(int n1, int* occ);
bool fused_in_kernel_halo(int n1);
cudaError_t fused_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1);
// the fused kernel alone (halo buffer already filled, or flag mode)
cudaError_t fused_kernel_launch(int n1, const FusedBatch& fb, int grid, cudaStream_t s);
// copies halo parts k0 .. k0 + nk - 1 (0-4: E1 E2 E3 B1 B3 of row p0 - 1; 5, 6: E1 E3 of row p1)
// of the work items into the halo buffer
cudaError_t halo_parts(int n1, const FusedBatch& fb, int k0, int nk, cudaStream_t s);
// one launch copying n rows (row i: tasks[i].n floats, a multiple of 4, 16-byte aligned) from
// src to dst: the halo rows of every work item of a batch's fused groups at once
struct RowCopy { const float* src; float* dst; int n; int pad; };
cudaError_t copy_rows(const RowCopy* tasks, int n, cudaStream_t s);
hyb_status fused_host_advance(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3]);
std::vector<int4> fused_items(int inst, int n2, int n_strips);
FusedInst fused_inst(const hyb_grid* g);
hyb_status fused_set_strips(hyb_grid* g, int n_strips);

}  // namespace hyb
