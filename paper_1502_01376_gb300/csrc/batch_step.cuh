// batch_step.cuh -- host interface of the batched step as one persistent launch (batch_step.cu):
// the CTAs of the launch are split into roles, one per group of fused 2D grids with a common n1
// and one for the quasi-3D modes; every role runs the device code of its own kernels
// (tm_body.cuh, tmt_body.cuh, q3d_body.cuh) on its CTAs.
#pragma once
#include "fused_api.cuh"
#include "q3d_body.cuh"

namespace hyb {

// roles: the 2D groups n1 = 4096, 512, 1024, 2048, then the quasi-3D modes
enum : int { kRoleTM = 0, kRoleT32, kRoleT64, kRoleT128, kRoleQ3, kRoles };
inline int role_of_n1(int n1) {
    return n1 == 4096 ? kRoleTM : n1 == 512 ? kRoleT32 : n1 == 1024 ? kRoleT64 : n1 == 2048 ? kRoleT128 : -1;
}

struct StepRole2D {
    int cta0 = 0, ncta = 0;        // CTAs [cta0, cta0 + ncta) of the launch (ncta = 0: no such group)
    FusedBatch fb;                 // the group's grids and work items (halo-buffer mode)
    const RowCopy* halo = nullptr; // the halo rows of the group's work items, copied by the role first
    int n_halo = 0;
};

struct StepArgs {
    StepRole2D r2[4];              // indexed by kRoleTM .. kRoleT128
    Q3Args q3;                     // the quasi-3D modes: CTAs [q3_cta0, q3_cta0 + q3_ncta)
    int q3_cta0 = 0, q3_ncta = 0;
    int* q3_err = nullptr;         // bounded waits of the quasi-3D role report here
    unsigned* sync = nullptr;      // [kRoles][2] role barriers: arrive counter, generation (zeroed once)
    // optional (autotuner): per role the earliest start and latest end of its CTAs (%globaltimer, ns);
    // [kRoles][2], set to {max, 0} before the launch
    unsigned long long* stamp = nullptr;
};

size_t batch_step_smem_bytes();
// CTAs of the launch: one per SM (every CTA must be resident: the roles have grid-wide barriers)
cudaError_t batch_step_ctas(int* n);
cudaError_t batch_step_launch(const StepArgs& a, int grid, cudaStream_t s);
// self-test of the role barrier's bounded wait (sync: two zeroed words)
cudaError_t role_probe(unsigned* sync, int* err, long long limit, cudaStream_t s);

}  // namespace hyb
