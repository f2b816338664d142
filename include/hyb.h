/*
 * hyb.h -- C ABI of libhyb.so, the GB300 (sm_103a) implementation of the
 * hybrid Yee-FFT Maxwell field advance of Yu et al., arXiv:1502.01376
 * ("Mitigation of numerical Cerenkov radiation and instability using a hybrid
 * finite difference-FFT Maxwell solver and a local charge conserving current
 * deposit").
 *
 * Conventions shared by every call
 * --------------------------------
 * Fields are real arrays of the grid's precision (float for precision 32,
 * double for 64), row-major [n3][n2][n1] (n3 = 1 in 2D), x1 contiguous,
 * 16-byte aligned, resident in this process's current CUDA device memory
 * unless a call says "host".  A half-integer position i+1/2 is stored at
 * index i (Yee staggering, Sec. 2.1): E1(i1+1/2,i2), E2(i1,i2+1/2), E3(i1,i2),
 * B1(i1,i2+1/2), B2(i1+1/2,i2), B3(i1+1/2,i2+1/2), j like E, rho at integer
 * points; 3D adds the standard Yee offsets in x3 (Sec. 2.4).  All boundaries
 * are periodic.  Units: c = 1; Ampere's law carries `ampere` (4 pi) times j.
 *
 * Ownership: field, current, charge and particle memory belongs to the
 * caller; the library borrows the pointers given to hyb_bind_fields until the
 * next bind or hyb_destroy_grid.  The library owns its mode tables and its
 * scratch, allocated in hyb_create_grid.
 *
 * Streams: every call is enqueued on the grid's stream and returns without
 * waiting, except hyb_diag, hyb_advance_host, hyb_check and
 * hyb_destroy_grid, which synchronise that stream.
 *
 * Errors: no call throws, exits or aborts.  A non-zero hyb_status is
 * returned and hyb_last_error() gives a one-line message (thread-local).
 * Kernels that detect bad input at run time (a particle moving a cell or more
 * in one step) record it in a device flag that hyb_check reports.
 */
#ifndef HYB_H_
#define HYB_H_

#include <stdint.h>

#if defined(__GNUC__)
#define HYB_API __attribute__((visibility("default")))
#else
#define HYB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hyb_grid hyb_grid;   /* opaque */

typedef enum {
    HYB_OK = 0,
    HYB_EINVAL = 1,     /* bad argument, size or unsupported combination */
    HYB_ECOURANT = 2,   /* dt above the Courant limit of Sec. 2.2 */
    HYB_EALIGN = 3,     /* pointer not 16-byte aligned */
    HYB_ECUDA = 4,      /* a CUDA runtime call failed */
    HYB_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    HYB_ESTATE = 6,     /* call out of order (e.g. fields not bound) */
    HYB_ENOMEM = 7,     /* device allocation failed */
    HYB_EDATA = 8       /* a kernel rejected input data (see hyb_check) */
} hyb_status;

typedef struct {
    int dims;             /* 2, 3, or 20 for quasi-3D (one azimuthal mode; see azimuthal_m) */
    int n1, n2, n3;       /* grid points along x1 (FFT, even, power of two), x2, x3 (FD); n3 ignored in 2D */
    double dx1, dx2, dx3; /* cell sizes */
    double dt;            /* time step; must satisfy the Courant limit of Sec. 2.2 */
    int precision;        /* 32 (float fields) or 64 (double fields) */
    int correct_j1;       /* 1: apply Eq. currentcorrection to j1 inside hyb_advance */
    double filt_kc;       /* k1 low-pass filter of Sec. 4 on j: centre, fraction of pi/dx1; on iff 0 < filt_kc < 1 */
    double filt_w;        /* filter transition width, fraction of pi/dx1 (raised cosine, F(kc) = 1/2) */
    double kmod_l, kmod_u;/* dispersion bump of Sec. 4: k1 range, fractions of k_g1 = 2 pi/dx1 */
    double kmod_max;      /* bump height, fraction of k_g1; 0 = off */
    int yee_mode;         /* 1: [k]1 = sin(k1 dx1/2)/(dx1/2) (recovers the Yee solver, Sec. 2.1) */
    double ampere;        /* coefficient of j in Ampere's law; 0 selects 4 pi */
    int path;             /* 0: fastest available, as measured on GB300 (fused where it applies,
                                else path 1, faster than path 3 at every n1 measured);
                             1: three-pass (FFT, update, inverse FFT);
                             2: fused single-pass (precision 32, dims 2, n1 in 512..4096);
                             3: three-pass with the x1 transform as a dense DFT matrix product on
                                the tensor cores (tcgen05), FP32 split into BF16 hi + lo (3
                                products), FP32 accumulation (precision 32, dims 2 or 3,
                                16 <= n1 <= 1024); about 1e-5 relative error per field;
                             4: as 3 with FP32 split into three BF16 parts (6 products): the
                                error of the FP32 radix path */
    int azimuthal_m;      /* dims 20 only: azimuthal mode number 0 <= m <= 64.  The grid is then
                             (z, r) = (x1, x2) with n1 = nz, n2 = nr <= 65535, dx1 = dz, dx2 = dr, a
                             perfectly conducting wall at r = n2 dx2, the axis at r = 0, and
                             every field and current is COMPLEX (interleaved re, im) of the
                             grid's precision: the amplitude of exp(i m phi) (Sec. 5). */
} hyb_grid_desc;

/* Courant limit dt_max = 2 / sqrt(pi^2/dx1^2 + 4/dx2^2 [+ 4/dx3^2]) of Sec. 2.2;
 * for a quasi-3D mode m, 4/dx2^2 is replaced by (4 m^2 + 6)/dx2^2, a bound on
 * the largest eigenvalue of the cylindrical radial operator (at the axis). */
HYB_API double hyb_courant_limit(const hyb_grid_desc* desc);

/* Validates desc (sizes, Courant limit -> HYB_ECOURANT, precision/path
 * combination), computes the per-mode tables of Eqs. currentcorrection and
 * hybrid2db1-hybrid2de3 and the Sec. 4 filter/bump in FP64 on the host, rounds
 * them once to the run precision, uploads them and allocates scratch on the
 * current device.  stream is a cudaStream_t (NULL = legacy default stream). */
HYB_API hyb_status hyb_create_grid(const hyb_grid_desc* desc, void* stream, hyb_grid** out);

/* Replaces the stream later calls are enqueued on. */
HYB_API hyb_status hyb_set_stream(hyb_grid* g, void* stream);

/* Borrows the caller's device arrays: E[3], B[3], J[3] (required, each
 * n1*n2*n3 elements of the grid's precision) and rho (nullable; used only by
 * hyb_diag's Gauss residual).  Checks 16-byte alignment (HYB_EALIGN). */
HYB_API hyb_status hyb_bind_fields(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3], void* rho);

/* Sec. 2.3 charge-conserving (Esirkepov-form) deposit of j^{n+1/2} into the
 * bound J (zeroed first) for np particles moving from x^n to x^{n+1}:
 *   cell    int32 [np][dims]: integer cell of x^n along each axis (0 <= c < n);
 *   off_old real  [np][dims]: x^n  - cell, in cell units, in [0, 1);
 *   off_new real  [np][dims]: x^{n+1} - cell, in cell units, |off_new - off_old| < 1;
 *   v3      real  [np] (2D only, nullable): out-of-plane velocity for j3;
 *   q       real  [np]: macro-particle charge;
 *   shape_order 1 (linear), 2 (quadratic) or 3 (cubic) B-spline.
 * Real arrays are of the grid's precision, device resident.  Particles that
 * break the range conditions are skipped and flagged (hyb_check -> HYB_EDATA). */
HYB_API hyb_status hyb_deposit(hyb_grid* g, const int32_t* cell, const void* off_old, const void* off_new,
                       const void* v3, const void* q, int64_t np, int shape_order);

/* Field gather and relativistic Boris push of np particles, the step that feeds
 * hyb_deposit.  Gather: the momentum-conserving interpolation of the Appendix
 * (Eqs. for S_E and S_B): each component of E and B is interpolated with the
 * order-l shape s_l along every axis, from its own staggered grid (2D: E1 at
 * (i1+1/2, i2), E2 (i1, i2+1/2), E3 (i1, i2), B1 (i1, i2+1/2), B2 (i1+1/2, i2),
 * B3 (i1+1/2, i2+1/2); 3D as in the 3D Yee cell).  Push (c = 1, Gaussian units,
 * u = gamma v): the Boris rotation, h = (q/m) dt/2,
 *   u- = u + h E;  t = h B / gamma(u-);  s = 2 t / (1 + t.t);
 *   u+ = u- + (u- + u- x t) x s;  u^{n+1/2} = u+ + h E;
 *   x^{n+1} = x^n + dt u^{n+1/2} / gamma(u^{n+1/2}).
 * E and B are read from the bound arrays, which the caller holds at the
 * particles' time level n (E^n and, e.g., the mean of B^{n-1/2} and B^{n+1/2}).
 *   cell    int32 [np][dims] in/out: the cell the offsets refer to (0 <= c < n);
 *   off     real  [np][dims] in/out: x^n - cell in cell units, in [-1, 2) on entry
 *           (a previous step's off_new); the call first moves each particle to
 *           the cell that holds it (periodic), so that on exit 0 <= off < 1;
 *   u       real  [np][3] in/out: u^{n-1/2} on entry, u^{n+1/2} on exit;
 *   qm      real  [np]: charge-to-mass ratio q/m;
 *   off_new real  [np][dims] out: x^{n+1} - cell (cell units), hyb_deposit's off_new;
 *   v3      real  [np] out, nullable, 2D only: u3/gamma, hyb_deposit's v3;
 *   shape_order 1, 2 or 3.
 * Real arrays are of the grid's precision, device resident; fields periodic.
 * 2D: cell, off and off_new must be aligned to one particle's pair (8 bytes,
 * 2 reals), else HYB_EALIGN.
 * Particles with a cell out of range or an offset outside [-1, 2) are left
 * unchanged (off_new = off) and flagged (hyb_check -> HYB_EDATA). */
HYB_API hyb_status hyb_push(hyb_grid* g, int32_t* cell, void* off, void* u, const void* qm, void* off_new, void* v3,
                            int64_t np, int shape_order);

/* ---------------------------------------------------------------------------
 * The particle-in-cell loop around the advance (the drifting-plasma runs whose
 * measured NCI growth Sec. 4 reports): E at integer steps, B at half steps
 * (Sec. 2.1), the charge-conserving current of Sec. 2.3, and the particle step
 * the Appendix's dispersion relation assumes (fields gathered at the
 * particles' time level with B time-centred, momentum-conserving
 * interpolation).  Per step, with E = E^n, B = B^{n-1/2} bound to g and the
 * particles at x^n with u^{n-1/2}:
 *   B^n = (B^{n-1/2} + B^{n+1/2})/2, B^{n+1/2} from Faraday's update of a copy;
 *   hyb_push with E^n, B^n (u^{n+1/2}, x^{n+1});  hyb_deposit (j^{n+1/2});
 *   hyb_advance (E^{n+1}, B^{n+1/2});  off <- off_new.
 * hyb_pic_create borrows g (which must stay bound to the same arrays) and
 * allocates a second grid of the same description and 9 scratch fields.
 * When g is k1-resident (hyb_set_resident) the step takes B^n from the
 * resident spectra instead (B^{n-1/2} + Faraday(E^n)/2 per mode, transformed
 * into scratch), and its advance transforms only j forward: 12 row transforms
 * per step instead of two full advances. */
typedef struct hyb_pic hyb_pic;   /* opaque */
HYB_API hyb_status hyb_pic_create(hyb_grid* g, hyb_pic** out);

/* nsteps PIC steps on the grid's stream (asynchronous).  Particle arrays as
 * for hyb_push and hyb_deposit (device, the grid's precision): cell int32
 * [np][dims], off [np][dims] (x^n on entry, x^{n+nsteps} on exit, in [-1, 2)
 * of its cell), u [np][3], qm [np] (q/m), q [np] (macro-particle charge),
 * off_new [np][dims] (scratch, ends equal to off), v3 [np] (scratch; required
 * in 2D).  Errors of the push and deposit are flagged as for them (hyb_check).
 * With nsteps >= 4 (and unless g's fused kernel exchanges halo rows inside
 * the launch, as at n1 = 4096, or the grid's stream is being captured by the
 * caller) the first step runs as plain
 * launches and the others replay one captured step as a CUDA graph on a
 * private stream ordered after and before the grid's stream; the graph is kept
 * for later calls with the same arrays.  Results agree with plain steps to
 * rounding (the deposit's atomic sums are not ordered). */
HYB_API hyb_status hyb_pic_step(hyb_pic* p, int32_t* cell, void* off, void* u, const void* qm, const void* q,
                                void* off_new, void* v3, int64_t np, int shape_order, int nsteps);

/* Frees the PIC step's second grid and scratch (not g). */
HYB_API hyb_status hyb_pic_destroy(hyb_pic* p);

/* Eq. currentcorrection alone, in place on the bound J1:
 * j1 <- IFFT_x1[ sin(k1 dx1/2)/(k1 dx1/2) FFT_x1[j1] ]. */
HYB_API hyb_status hyb_correct_current(hyb_grid* g);

/* The same j1 correction as hyb_correct_current, for callers that cannot
 * allocate device memory (the paper has no counterpart; this is a library
 * convenience).  It needs no grid: desc gives the sizes and cell size (dims,
 * n1, n2, n3, dx1, precision, yee_mode, kmod_l, kmod_u and kmod_max are read),
 * j1 is the caller's device array (in place), stream a cudaStream_t.  It
 * allocates nothing: its tables and the k1-space copy of a block of rows live
 * in one static 8 MiB device array of the library, which every GPU that loads
 * the library keeps until the process exits.  The tables are computed by a
 * kernel on the stream (no host-to-device copy).  Rows are processed in blocks
 * that fit the array; an n1 whose single row does not fit is rejected with
 * HYB_EINVAL.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call reuses the same array, so calls whose work overlaps on the GPU
 * (different streams, or different host threads) race: serialise them. */
HYB_API hyb_status hyb_correct_current_noalloc(const hyb_grid_desc* desc, void* j1, void* stream);

/* The Sec. 4 k1 low-pass form factor alone, in place on all three bound J components. */
HYB_API hyb_status hyb_filter(hyb_grid* g);

/* nsteps of the hybrid advance, Eqs. hybrid2db1-hybrid2de3 (3D: Sec. 2.4),
 * in place on the bound fields: on entry E = E^n, B = B^{n-1/2}, J = j^{n+1/2}
 * (the same J for every step); on exit E = E^{n+nsteps}, B = B^{n+nsteps-1/2}.
 * Per step: FFT along x1 of E, B, j; correction of j1 (if correct_j1) and the
 * filter of j (if on) in k1 space; Faraday then Ampere per k1 mode with
 * finite differences in x2 (and x3); inverse FFT. */
HYB_API hyb_status hyb_advance(hyb_grid* g, int nsteps);

/* k1-resident fields (on = 1) or not (on = 0, the default).  The method
 * applies every curl update to the x1-spectra of the fields (Sec. 2.1), and
 * the real-space fields are needed only where particles gather them, so with
 * on = 1 the grid keeps the k1-space E and B of its last step in its own
 * scratch and the next step transforms only j: per step one forward FFT of
 * the three j components, the same k1-space correction, filter, Faraday and
 * Ampere updates, and the inverse FFT of E and B into the bound arrays, which
 * thereby become an output (the fields to gather) rather than the input.  The
 * first step after this call, after hyb_bind_fields or inside
 * hyb_advance_host imports E and B from the bound (or host) arrays as a
 * normal step does; to feed changed real-space fields in later, call
 * hyb_set_resident(g, 1) again.  Results are those of hyb_advance up to the
 * rounding of the dropped inverse/forward round trip.  Resident grids run the
 * three-pass kernels (the fused single pass keeps no spectra); on a grid made
 * for the fused path the first call with on = 1 synchronises the grid's
 * stream and allocates the spectral state (9 n2 n3 (n1/2 + 1) complex values).
 * HYB_EINVAL for quasi-3D grids or on outside {0, 1}. */
HYB_API hyb_status hyb_set_resident(hyb_grid* g, int on);

/* The same as hyb_advance, but E, B, J are HOST arrays (pinned memory
 * recommended): they are copied into the bound device arrays, advanced, and
 * E, B are copied back.  Synchronises the grid's stream.  On the fused path
 * with nsteps = 1 the copies and the step are pipelined over chunks of rows
 * (the device arrays end up holding the same values). */
HYB_API hyb_status hyb_advance_host(hyb_grid* g, void* const E[3], void* const B[3], void* const J[3], int nsteps);

/* FP64 diagnostics of the bound fields, synchronous:
 *   out[0..5]  sum f^2 dV / (8 pi) of E1, E2, E3, B1, B2, B3;
 *   out[6]     max |div B|, div B = sigma+ B1 + d2+ B2 [+ d3+ B3] at the B-cell corners;
 *   out[7]     max |G|, G = sigma- E1 + d2- E2 [+ d3- E3] - ampere F rho (Sec. 2.3; F the
 *              current filter, rho taken as 0 if not bound);
 *   out[8]     rms of G. */
HYB_API hyb_status hyb_diag(hyb_grid* g, double out[9]);

/* Synchronises the grid's stream and reports (and clears) the device-side flag:
 * HYB_EDATA when hyb_deposit skipped out-of-range particles, HYB_ETIMEOUT when a
 * bounded device wait of the fused advance (halo flag or row staging) gave up;
 * otherwise HYB_OK. */
HYB_API hyb_status hyb_check(hyb_grid* g);

/* Self-test of the bounded device-side waits (the paper has no counterpart).
 * Runs one probe kernel that waits on a condition nothing satisfies, with the
 * same wait code the fused advance uses: which = 0, the release/acquire flag
 * wait of the in-kernel halo exchange; which = 1, the mbarrier wait of the row
 * staging; which = 2, the barrier between the CTAs of a role of the
 * single-launch batched step (a role of two CTAs, one of which never arrives).
 * The limit is `seconds` at the device's clock rate.  Returns HYB_ETIMEOUT
 * when the wait gave up as designed (the expected result), HYB_OK if the
 * condition was met, HYB_EINVAL for which not in {0, 1, 2} or seconds not in
 * (0, 10], HYB_ECUDA on a CUDA error.  Synchronous on `stream`; allocates and
 * frees three ints of device memory. */
HYB_API hyb_status hyb_wait_selftest(int which, double seconds, void* stream);

/* Frees the grid's tables and scratch (not the caller's arrays). NULL is a no-op. */
HYB_API hyb_status hyb_destroy_grid(hyb_grid* g);

/* Message for the last failing call on this thread ("" if none). */
HYB_API const char* hyb_last_error(void);

/* Instrumentation: start and stop are cudaEvent_t handles (NULL disables).
 * While set, every step of hyb_advance records start immediately before and
 * stop immediately after the launch of its dominant kernel (the fused kernel
 * on path 2; the whole step on path 1), on the grid's stream, so a caller can
 * time that kernel alone.  The events are borrowed, not owned. */
HYB_API hyb_status hyb_set_kernel_events(hyb_grid* g, void* start, void* stop);

/* ---------------------------------------------------------------------------
 * Batches: many independent grids advanced together (the paper applies the
 * solver to many grid geometries; batching them is this library's design).
 * Grids on the fused path are grouped by n1 and cut into (grid, strip) work
 * items; quasi-3D FP32 modes with nz = 2048 and a common radial grid are
 * advanced together.  One step of all grids is captured once in a CUDA graph
 * and replayed by hyb_batch_advance.  The step is either
 *   - ONE persistent cooperative launch (one 768-thread CTA per SM) whose CTAs
 *     are split into roles: one per n1 group (n1 = 512, 1024, 2048, 4096),
 *     which copies its halo rows and sweeps its work items, and one for the
 *     quasi-3D modes, which runs their z transforms, leapfrog and inverse
 *     transforms with barriers of its own CTAs between them.  Available when
 *     every grid of the batch belongs to such a role (at most 8 quasi-3D
 *     modes); the default then.
 *   - a graph of launches: per group one persistent launch after one copy of
 *     all groups' halo rows, three launches per 8 quasi-3D modes, and each
 *     other grid's own step, on forked streams.
 * Both give the same bits.
 * ------------------------------------------------------------------------- */
typedef struct hyb_batch hyb_batch;   /* opaque */

/* Creates n grids (each as hyb_create_grid would, on the same stream). */
HYB_API hyb_status hyb_batch_create(const hyb_grid_desc* descs, int n, void* stream, hyb_batch** out);

/* Binds grid i of the batch to caller device arrays (as hyb_bind_fields; no rho). */
HYB_API hyb_status hyb_batch_bind(hyb_batch* b, int i, void* const E[3], void* const B[3], void* const J[3]);

/* Autotuner: for each group, times `trials` launches for each candidate strip
 * height (rows per work item) on scratch fields it allocates and frees, each
 * after a write larger than the L2 (a group's data arrives cold inside a
 * step), and keeps the fastest.  Then, when the single launch is available
 * and every grid is bound: rounds of (each group's strip height for the
 * current split, then CTAs in proportion to the CTA time each role took in
 * timed launches, up to 6 rounds), then one-CTA moves to the roles that
 * finish last while the launch gets faster, keeping the fastest split and
 * heights; finally the faster of the single launch and the graph of launches
 * (each timed as a graph, `trials` steps after L2 flushes).  These runs
 * advance the bound fields, which are saved first (device copies of every
 * grid's E and B, allocated and freed here) and restored after, so the fields
 * end as they were.  Synchronises. */
HYB_API hyb_status hyb_batch_tune(hyb_batch* b, int trials);

/* nsteps of every grid of the batch, one CUDA-graph launch per step, with the
 * same state contract as hyb_advance.  The graph is (re)captured on the first
 * call after a bind or a tune. */
HYB_API hyb_status hyb_batch_advance(hyb_batch* b, int nsteps);

/* Tuned rows per strip of the group with this n1 (0 if none). */
HYB_API int hyb_batch_rows_per_strip(const hyb_batch* b, int n1);

/* Sets the rows per strip of the group with this n1 (as the autotuner would),
 * e.g. to reuse a height found by an earlier hyb_batch_tune.  h >= 1.
 * HYB_EINVAL if no group has this n1.  Synchronous (uploads the work items). */
HYB_API hyb_status hyb_batch_set_rows_per_strip(hyb_batch* b, int n1, int h);

/* Kernel launches in one step of the batch (the nodes of its graph). */
HYB_API int hyb_batch_launches_per_step(const hyb_batch* b);

/* Chooses the form of the step: on != 0 the single persistent launch
 * (HYB_EINVAL if some grid has no role in it), 0 the graph of launches.
 * Takes effect at the next hyb_batch_advance (re-capture). */
HYB_API hyb_status hyb_batch_set_single_launch(hyb_batch* b, int on);

/* 1 if a step is the single persistent launch, else 0. */
HYB_API int hyb_batch_single_launch(const hyb_batch* b);

/* hyb_check of every grid of the batch (synchronises the batch's stream, reads
 * and clears each grid's device-side flag): HYB_ETIMEOUT when a bounded wait of
 * a step gave up (a role barrier of the single launch, a row staging or halo
 * wait), HYB_EDATA for a deposit's skipped particles; the first error found is
 * returned and described by hyb_last_error. */
HYB_API hyb_status hyb_batch_check(hyb_batch* b);

/* CTAs of role r of the single launch (0: n1 = 4096, 1: 512, 2: 1024,
 * 3: 2048, 4: the quasi-3D modes); 0 if the role is absent or the single
 * launch is not available. */
HYB_API int hyb_batch_role_ctas(const hyb_batch* b, int r);

/* Sets the CTAs of the single launch's roles (ctas[0..4], as hyb_batch_role_ctas
 * numbers them), e.g. to reuse a split found by an earlier hyb_batch_tune:
 * at least one CTA for every role the batch has, zero for the others, at most
 * one CTA per SM in all.  HYB_EINVAL otherwise or without a single launch. */
HYB_API hyb_status hyb_batch_set_role_ctas(hyb_batch* b, const int* ctas);

/* Duration (ms, first CTA start to last CTA end) of role r in the fastest
 * single launch hyb_batch_tune timed; 0 before a tune or for an absent role. */
HYB_API double hyb_batch_role_ms(const hyb_batch* b, int r);

/* Frees the batch and its grids (not the caller's arrays). */
HYB_API hyb_status hyb_batch_destroy(hyb_batch* b);

/* ---------------------------------------------------------------------------
 * NCI analysis (Sec. 3 and the Appendix): growth rate of the numerical
 * Cerenkov instability of a cold plasma drifting along x1 on the hybrid
 * solver's grid, from the roots of the numerical dispersion relation
 * (Eq. 2dmodesres with its coupling term; hybrid operators [k]E1 = [k]B1 = k1
 * plus the Sec. 4 bump, [k]E2 = [k]B2 = sin(k2 dx2/2)/(dx2/2); B time-centred,
 * S_B3 = S'_B3 cos(omega dt/2), as the cubic Eq. asym1 implies), in FP64 on the
 * GPU.  The roots of an alias are ALL zeros of [omega] D(omega) (omega' - k1' v0)
 * in the disk |omega - omega_res| < (wp2/gamma)^(1/3) about the beam resonance
 * omega' = k1' v0: counted by the argument principle on the disk's circle,
 * located by deflated Newton iterations from the cubic's roots and rings of
 * seeds, and, when seeds leave some unfound, by argument-principle subdivision.
 *   samples  device double [n][12]: dt, dx1, dx2, gamma, wp2 (plasma frequency^2,
 *            n/n_p), filt_kc, filt_w (current filter, fractions of pi/dx1;
 *            kc outside (0,1) = off), k1, k2, kmod_l, kmod_u, kmod_max (Sec. 4
 *            k1 modification, fractions of 2 pi/dx1; kmod_max = 0 = off);
 *   order    particle shape order l (1..3), momentum-conserving interpolation;
 *   correct_j1  1: the Eq. currentcorrection factor multiplies S_j1;
 *   alias    device int [n_alias][2]: (mu, nu1) pairs;
 *   growth   device double [n][n_alias]: max Im(omega) over the roots of that
 *            alias (0 if none grows);
 *   root     device double [n][n_alias][2] (nullable): the root that gives it.
 * Asynchronous on stream. */
HYB_API hyb_status hyb_nci_growth(const double* samples, int64_t n, int order, int correct_j1,
                                  const int* alias, int n_alias, double* growth, double* root, void* stream);

/* The same root sets in full (the Appendix relation, as hyb_nci_growth):
 *   roots    device double [n][n_alias][max_roots][2]: the zeros in the disk,
 *            unordered, zero-filled after count;
 *   count    device int [n][n_alias]: how many were found;
 *   growth   device double [n][n_alias] as in hyb_nci_growth;
 *   err      device int (nullable), OR-ed: 1 = more than 16 zeros in a disk
 *            (the rest dropped), 2 = a count the argument principle could not
 *            resolve (a zero on a contour after every refinement).
 * Asynchronous on stream. */
HYB_API hyb_status hyb_nci_roots(const double* samples, int64_t n, int order, int correct_j1, const int* alias,
                                 int n_alias, int max_roots, double* roots, int* count, double* growth, int* err,
                                 void* stream);

/* ---------------------------------------------------------------------------
 * NCI surrogate: a small MLP (n_in -> width x depth tanh layers -> 1) trained
 * on the root solver's growth rates to pick the filter cutoff and time step
 * before a run.  Forward, backward and Adam are this library's kernels: BF16
 * weights and activations as tensor-core operands (tcgen05.mma), FP32
 * accumulation, FP32 master weights.  Parameters are laid out per layer as
 * W[out][in] then b[out] (FP32).  x is device FP32 [B][n_in]; targets, outputs
 * device FP32 [B].
 * ------------------------------------------------------------------------- */
typedef struct hyb_mlp hyb_mlp;   /* opaque */

/* init_params: host FP32 [hyb_mlp_num_params] (NULL = zeros). Synchronous. */
HYB_API hyb_status hyb_mlp_create(int n_in, int width, int depth, const float* init_params, hyb_mlp** out);
HYB_API int64_t hyb_mlp_num_params(const hyb_mlp* m);
HYB_API hyb_status hyb_mlp_set_params(hyb_mlp* m, const float* params_host);
HYB_API hyb_status hyb_mlp_get_params(hyb_mlp* m, float* params_host);
/* y = network(x), asynchronous on stream. */
HYB_API hyb_status hyb_mlp_forward(hyb_mlp* m, const float* x, int64_t B, float* y, void* stream);
/* Gradient of the mean-squared error sum_b (y_b - t_b)^2 / B with respect to
 * every parameter (host FP32 [num_params], nullable) and the loss (host,
 * nullable); synchronises stream.  Used to check the backward kernels. */
HYB_API hyb_status hyb_mlp_gradients(hyb_mlp* m, const float* x, const float* target, int64_t B, float* grad_host,
                                     float* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean-squared error;
 * the loss before the step is written to loss_dev (device FP32, nullable). */
HYB_API hyb_status hyb_mlp_train_step(hyb_mlp* m, const float* x, const float* target, int64_t B, float lr, float* loss_dev,
                                      void* stream);
/* Kernels this network has launched so far (instrumentation: a training step
 * of L = depth + 1 layers launches 3 L (one GEMM per layer forward, two per
 * layer backward but one for the first layer, the Adam step), a forward pass L). */
HYB_API int64_t hyb_mlp_launch_count(const hyb_mlp* m);
HYB_API hyb_status hyb_mlp_destroy(hyb_mlp* m);

/* Which advance path a grid runs: 1 three-pass, 2 fused, 3 and 4 three-pass with DFT-GEMM
 * (2 and 3 BF16 parts). */
HYB_API int hyb_grid_path(const hyb_grid* g);

/* Name of the kernel that does a step's work on this grid's path (the fused kernel's name
 * on path 2; a description of the step on the others).  A static string owned by the
 * library; "" for a null grid. */
HYB_API const char* hyb_step_kernel(const hyb_grid* g);

/* Number of kernel launches one hyb_advance step of this grid issues. */
HYB_API int hyb_launches_per_step(const hyb_grid* g);

#ifdef __cplusplus
}
#endif

#endif /* HYB_H_ */
