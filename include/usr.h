/*
 * usr.h -- C ABI of libusr: u-series electrostatic energy, forces and
 * potentials for point charges in an orthorhombic periodic box, evaluated on
 * one NVIDIA GB300 (sm_103a) GPU.
 *
 * Method: Predescu et al., "The u-series: a separable decomposition for
 * electrostatics computation with improved accuracy", arXiv:1911.01377.
 *   E = E_near + E_far + E_self                          (Eq. 3 with Eqs. 19-22)
 *   E_near = 1/2 sum_{i != j, images} q_i q_j N(r_ij), N(r) = 1/r - F(r) for
 *            r < r_c and 0 beyond                          (Eq. 20)
 *   E_far  = far part, the Gaussians of F(r) summed over all periodic images
 *            with the k = 0 term dropped (Eqs. 4, 9); evaluated by Gaussian
 *            charge spreading onto a grid, three per-axis 1D convolutions per
 *            Gaussian term (Eqs. 31-32, Sec. V) and interpolation back to the
 *            charges; N terms kept by the bound of Eq. 33
 *   E_self = -1/2 F(0) sum q_i^2                           (Eq. 10's self term)
 * Units: charges in e, lengths in Angstrom, Coulomb constant 1 (energies in
 * e^2/Angstrom, forces in e^2/Angstrom^2, potentials in e/Angstrom).
 *
 * Conventions for every entry point:
 *   - All pointers are owned by the caller; the library never frees them.
 *   - "device" pointers must be CUDA device (or managed) memory on the
 *     context's device; "host" pointers ordinary host memory (pinned memory
 *     makes the copies asynchronous and faster).
 *   - Position/charge and output arrays are float4-packed (x, y, z, q) and
 *     (Fx, Fy, Fz, phi) rows, n rows, 16-byte aligned.
 *   - Positions may lie outside the box; they are wrapped periodically.  The
 *     single-precision wrap is exact within 2^22 box lengths of the box; a
 *     row it cannot bring into the box is evaluated as a zero charge at the
 *     origin and reported as USR_ERR_NONFINITE, like a non-finite row.
 *   - Work is enqueued on the given CUDA stream (cudaStream_t passed as void*,
 *     NULL = legacy default stream) and returns before the GPU finishes,
 *     except where an entry point says it synchronises.  A context must not
 *     be used from two host threads or on two streams at the same time.
 *   - No entry point throws, traps or aborts.  Problems found on the GPU
 *     (non-finite inputs) set a status word read by usr_last_device_status.
 */
#ifndef USR_H
#define USR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    USR_OK = 0,
    USR_ERR_ARG = 1,        /* null or misaligned pointer, n < 0, unknown enum value */
    USR_ERR_BOX = 2,        /* geometry the GPU path does not support (see usr_plan) */
    USR_ERR_NONFINITE = 3,  /* a coordinate or charge was NaN or infinite, a position lay too far from
                               the box to be wrapped, or a near-part sum left the fixed-point range
                               (two charges at one point) (found on the GPU) */
    USR_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    USR_ERR_OOM = 5,        /* device memory allocation failed */
    USR_ERR_TIMEOUT = 6,    /* a bounded device wait ran out */
    USR_ERR_CAPACITY = 7,   /* more atoms than the context was created for */
    USR_ERR_INTERNAL = 8    /* a device-side consistency check failed (a library bug; results invalid) */
} usr_status;

/*
 * Arithmetic of the per-axis far-part convolutions (Sec. V).  The split forms
 * run on the tensor cores (tcgen05): every operand is split into a high and a
 * low part and three products (hi*hi + hi*lo + lo*hi) are accumulated in FP32.
 * They need every grid dimension to be a multiple of 4 (TF32X3) or 8 (BF16X3).
 */
typedef enum {
    USR_CONV_FP32 = 0,      /* FP32 CUDA-core GEMMs with FP32 accumulation */
    USR_CONV_TF32X3 = 1,    /* tensor cores, TF32 hi/lo split operands, FP32 accumulation */
    USR_CONV_BF16X3 = 2     /* tensor cores, BF16 hi/lo split operands, FP32 accumulation */
} usr_conv;

/* Presets: the parameter rows printed in Table 2 (b = 2) and Table 1. */
typedef enum {
    USR_PRESET_C0_B2 = 0,   /* Table 2 row 1: C0 construction, Eq. 19 */
    USR_PRESET_C1_B2 = 1,   /* Table 2 row 2: C1 construction, Eq. 24 (recommended, Sec. VI) */
    USR_PRESET_C2_B2 = 2,   /* Table 2 row 3: C2 construction, Eq. 28 */
    USR_PRESET_T1_A = 3,    /* Table 1 row 1: C2 point of the C1 family, b = 1.6298 */
    USR_PRESET_T1_B = 4,    /* Table 1 row 2: b = 1.3207 */
    USR_PRESET_T1_C = 5     /* Table 1 row 3: b = 1.2181 */
} usr_preset;

/*
 * One u-series construction.  The far function at sigma = r_c / r0 (Eq. 23) is
 *   F(r) = c [ w0 exp(-r^2 / (2 s0^2 sigma^2)) + sum_{j>=1} b^-j exp(-r^2 / (2 b^2j sigma^2)) ],
 *   c = 2 ln(b) / sqrt(2 pi sigma^2)                               (Eqs. 19, 24, 28)
 * (Eq. 28's narrow term is taken unnormalised in s0: Table 2's third row
 * satisfies Eq. 27 only under that reading.)
 */
typedef struct {
    double b;          /* base; at least 1.0113, so that the full series down to amplitude
                          1e-20 of the first term has at most 4096 terms */
    double r0;         /* r_c / sigma */
    double w0;         /* weight of the narrowest Gaussian (1 for C0) */
    double s0;         /* width factor of the narrowest Gaussian (1 for C0, C1) */
    int n_terms;       /* Gaussians on the far grid (at most 16, and at most the terms of amplitude
                          >= 1e-20 of the first); 0 = smallest N whose Eq. 33 bound <= trunc_eps */
    double trunc_eps;  /* used when n_terms == 0; 0 means 1e-9 */
} usr_series;

typedef struct {
    double box[3];               /* box side lengths L_x, L_y, L_z (Angstrom, > 0, at most 1e5) */
    int grid[3];                 /* far-part grid points per axis (at most 4096, and at most
                                    2^31 - 1 in all) */
    double r_c;                  /* near-part cutoff; sigma = r_c / r0 */
    usr_series series;
    double spread_sigma_over_h;  /* spreading Gaussian width / largest grid spacing; 0 = 1.0 */
    int spread_points;           /* spreading stencil points per axis (even, 8..16); 0 = 12 */
    usr_conv conv;
    int max_atoms;               /* capacity of the context (rows per evaluation), at most 2^28 */
    int virial;                  /* 1: also compute the virial tensor (usr_virial); six more far-part
                                    convolution sets per evaluation */
    int multilevel;              /* 1: the wide Gaussian terms on a grid twice as coarse (Sec. V's remark
                                    that wider terms can be handled by multilevel summation): the terms
                                    whose deconvolved width is at least 2.25 coarse spacings on every axis
                                    are convolved on the coarse grid, reached from the fine grid and back
                                    by Gaussian restriction and prolongation (33 taps each way); with a
                                    tensor-core form the coarse passes run in TF32x3 whatever conv says
                                    (FP32 when a coarse extent is not a multiple of 4). Needs even grid
                                    sizes of at least 33 points per axis and virial = 0 (USR_ERR_BOX
                                    otherwise).  0: every term on the fine grid */
} usr_params;

/* Quantities derived from usr_params (all host-side, FP64). */
typedef struct {
    double sigma;          /* r_c / r0 */
    double F0;             /* F(0) of the full series, the self term constant */
    double spread_sigma;   /* sigma_s of the spreading Gaussian */
    double h[3];           /* grid spacings L / grid */
    double trunc_bound;    /* Eq. 33 bound for the chosen n_terms */
    int n_terms;           /* Gaussians of the far part (fine and coarse grids together) */
    int cells[3];          /* cell-list cells per axis, floor(L / r_c) */
    int poly_degree;       /* degree of the FP32 polynomial for the wide terms of F */
    int n_explicit;        /* leading Gaussians of F evaluated explicitly in the pair kernel */
    double poly_max_err;   /* max |error| of that polynomial on [0, r_c], relative to F(0) */
    double device_bytes;   /* usr_plan: device memory a new context for these parameters needs;
                              usr_info: device memory the context holds (its buffers only grow) */
    int n_terms_coarse;    /* of n_terms, those convolved on the coarse grid (multilevel = 1), else 0 */
} usr_plan_info;

/* Fill *out with a preset row (n_terms = 0, trunc_eps = 0).  Host only. */
usr_status usr_series_preset(int preset, usr_series* out);

/*
 * Validate parameters and derive the plan without touching the GPU.
 * USR_ERR_BOX when: any L, grid or r_c is non-positive; fewer than 3 cells
 * per axis (r_c > L/3); a grid axis has fewer than spread_points + 8 points;
 * the narrowest kept Gaussian is not wider than sqrt(2) sigma_s (Eq. 32's
 * deconvolved widths sqrt(sigma_j^2 - 2 sigma_s^2) must be real); or one
 * cell's spreading tile would exceed 112 KB of shared memory (cells of more
 * than about 15 grid points per side); or a split convolution form is asked
 * for on a grid whose dimensions are not multiples of 4 (TF32X3) or 8 (BF16X3);
 * or a grid beyond 4096 points per axis or 2^31 - 1 points in all; or a box
 * side beyond 1e5 Angstrom; or, with n_terms = 0, a bound of Eq. 33 that
 * needs more than 16 far terms (the small-b rows of Table 1 on boxes of
 * about 80 Angstrom and more: set n_terms, at most 16, to accept a larger
 * truncation error).
 * USR_ERR_ARG for null pointers or out-of-range series/stencil values;
 * USR_ERR_CAPACITY for max_atoms beyond 2^28; USR_ERR_OOM when the host runs
 * out of memory (no C++ exception crosses this interface).
 */
usr_status usr_plan(const usr_params* p, usr_plan_info* out);

typedef struct usr_ctx usr_ctx;

/*
 * Create a context on the current CUDA device: runs usr_plan, allocates all
 * device scratch for up to p->max_atoms atoms (owned by the context) and
 * uploads the tables.  Synchronises the device.  *out is NULL on failure.
 */
usr_status usr_init(const usr_params* p, usr_ctx** out);

/*
 * Point an existing context at another system (box, grid, cutoff, series,
 * spreading, convolution form, max_atoms): the plan is rebuilt on the host,
 * device buffers that are already large enough are reused, and the tables are
 * uploaded with asynchronous copies on `stream` (so evaluations enqueued after
 * it on the same stream see them).  Buffers too small for the new system are
 * reallocated, which synchronises the device; among systems no larger than
 * one the context has held before, nothing is allocated.  The paper has no
 * counterpart: this serves many independent systems from a pool of contexts.
 * Errors as usr_plan / usr_init; on error the context must be reconfigured
 * successfully or destroyed before further use.
 */
usr_status usr_reconfigure(usr_ctx* ctx, const usr_params* p, void* stream);

/* Free a context and its device memory (NULL is ignored).  Synchronises. */
void usr_destroy(usr_ctx* ctx);

/* Derived quantities of a context. */
usr_status usr_info(const usr_ctx* ctx, usr_plan_info* out);

/*
 * One evaluation, enqueued on `stream`, no host synchronisation, no
 * allocation (usable inside CUDA graph capture).
 *   xyzq   device, n rows (x, y, z, q) float32, caller order, read only
 *   out    device, n rows (Fx, Fy, Fz, phi) float32, caller order; F_i = -dE/dr_i,
 *          phi_i = dE/dq_i (the potential at i with i's self term included)
 *   energy device, 4 doubles: E, E_near, E_far, E_self (may be NULL)
 * n = 0 writes zero energies.  USR_ERR_CAPACITY if n > max_atoms.
 * Internally the far part runs on a second stream of the context, forked from
 * `stream` after the cell list and joined back before the near + far
 * combination, so the call stays ordered on `stream` (and capturable) as one
 * unit.  A context's buffers are reused by every call: calls on one context
 * from different streams must be ordered by the caller (an event between
 * them).  Cost: the cell list orders each cell by counting, quadratic in the
 * cell's occupancy, and the near part grows with the pairs inside r_c; at the
 * densities the method is made for (about 0.1 charges per cubic Angstrom)
 * cells hold tens to a few hundred atoms, while charges piled into one cell
 * make both stages slow.
 */
usr_status usr_eval(usr_ctx* ctx, int n, const float* xyzq, float* out, double* energy, void* stream);

/*
 * The same evaluation from host memory: copies xyzq (host) to the device,
 * evaluates, copies out (host) and energy (host, 4 doubles, may be NULL)
 * back, then synchronises `stream`.
 */
usr_status usr_eval_host(usr_ctx* ctx, int n, const float* xyzq, float* out, double* energy, void* stream);

/*
 * usr_eval_host without the final synchronisation: the copies and the
 * evaluation are enqueued on `stream` and the call returns at once.  xyzq,
 * out and energy (host, 4 doubles, may be NULL) must stay valid and unread
 * until the stream reaches this point (record an event after the call);
 * pinned host memory makes the copies asynchronous.
 */
usr_status usr_eval_host_async(usr_ctx* ctx, int n, const float* xyzq, float* out, double* energy, void* stream);

/*
 * Synchronise the context's last stream and return the device status of the
 * evaluations since the previous call, then clear it: USR_OK;
 * USR_ERR_NONFINITE (a non-finite position or charge, a position too far
 * from the box to be wrapped, or a near-part sum beyond the pair kernel's
 * fixed-point range of +-2^30 per part, as two charges at one point give);
 * USR_ERR_TIMEOUT (a bounded wait of the tensor-core convolution ran out and
 * the pass returned early, its output is not valid); USR_ERR_INTERNAL (a
 * kernel's own consistency check failed).  When several are set, that order
 * decides.
 */
usr_status usr_last_device_status(usr_ctx* ctx);

/* ---- serving: continuous batching of independent systems ------------- */

/*
 * A server evaluates a stream of independent systems (each its own box, grid,
 * cutoff and charges) on the current device.  Requests are queued by
 * usr_server_submit from any host thread; `slots` concurrent evaluation
 * slots, each a context with its own CUDA stream and its own host thread,
 * take them in arrival order as soon as a slot is free, and admit each once
 * the device memory all slots hold stays within hbm_budget_bytes.  The host
 * work of a request (its FP64 plan, table uploads, launches) runs on its
 * slot's thread, in parallel with the other slots; requests that arrive while
 * others run are admitted as slots and memory free up, and their device work
 * overlaps on the GPU.  A slot's context is re-targeted to each request
 * with usr_reconfigure, so cell lists, grids and tables stay resident and are
 * reused; memory is allocated only when a request is larger than anything
 * its slot held before.  The paper has no counterpart: it describes the
 * method for one system.
 */
typedef struct usr_server usr_server;
typedef struct {
    double hbm_budget_bytes;   /* device memory all slots may hold; 0 = 16 GiB */
    int slots;                 /* evaluations in flight at once (1..64); 0 = 8 */
} usr_server_params;

usr_status usr_server_create(const usr_server_params* p, usr_server** out);

/*
 * Queue one evaluation: p describes the system (p->max_atoms >= n), xyzq is
 * host memory (n rows x, y, z, q), out (n rows Fx, Fy, Fz, phi) and energy
 * (4 doubles, may be NULL) host memory the server writes.  All three must
 * stay valid until the request completes; pinned memory lets the copies
 * overlap.  *ticket identifies the request.  Thread-safe.
 */
usr_status usr_server_submit(usr_server* s, const usr_params* p, int n, const float* xyzq, float* out,
                             double* energy, long long* ticket);

/*
 * Move up to max completed requests out of the server: their tickets, the
 * latency from submission to results in host memory (ms) and their status
 * (USR_OK, or why the request failed: USR_ERR_OOM if it can never fit the
 * budget, a plan error, a device status).  Returns the number written.
 */
int usr_server_poll(usr_server* s, long long* tickets, double* latency_ms, int* status, int max);

/* Block until every submitted request has completed (timeout_s <= 0: no limit). */
usr_status usr_server_wait(usr_server* s, double timeout_s);

/* Device bytes the slots hold, requests waiting for admission, requests on the device. */
usr_status usr_server_info(usr_server* s, double* held_bytes, long long* queued, long long* in_flight);

/* Finish the queued requests, then free every slot (NULL is ignored). */
void usr_server_destroy(usr_server* s);

/* Static description of a status code. */
const char* usr_status_string(usr_status s);

/* ---- inspection entry points used by the parity tests ---------------- */

/*
 * Bin and sort only (the cell list of the near part).  Device outputs:
 *   cell       n ints, cell id of each atom (caller order), id = (cz*ny + cy)*nx + cx
 *   perm       n ints, caller index of the atom at each sorted position
 *              (sorted by cell, then by caller index)
 *   cell_start ncell + 1 ints, first sorted position of each cell
 *   xw         n rows float4 in sorted order: wrapped x, y, z and q
 * The cell predicate is the single-precision one documented in the oracle.
 */
usr_status usr_debug_cells(usr_ctx* ctx, int n, const float* xyzq, int* cell, int* perm,
                           int* cell_start, float* xw, void* stream);

/*
 * Pair list of the near part, summarised per atom (caller order): the number
 * of partners j != i with r^2 < r_c^2 under the single-precision predicate,
 * and the wrap-around sum of splitmix64(j) over them (j = caller index).
 */
usr_status usr_debug_pairs(usr_ctx* ctx, int n, const float* xyzq, int* count, uint64_t* hash,
                           void* stream);

/*
 * The cell list of usr_debug_cells without a context and without any device
 * allocation, for callers that cannot call cudaMalloc when they need it (a
 * host application that owns all GPU memory through a fixed pool, code that
 * runs inside allocator callbacks or builds CUDA graphs by hand, a tool
 * injected into another program that must not change its memory footprint).
 * The paper has no counterpart: this is a deployment variant of the cell-list
 * step of the near part.
 *   box        host, 3 doubles: box side lengths (> 0)
 *   cells      host, 3 ints: cells per axis (>= 1), at most 65,536 cells in all
 *   xyzq       device, n rows float4 (x, y, z, q), caller order, n <= 262,144
 *   cell, perm, cell_start, xw   device outputs, the same as usr_debug_cells
 *              (cell_start has cells[0]*cells[1]*cells[2] + 1 ints)
 * The counting sort's temporaries live in one fixed file-scope device array
 * of about 6.3 MB, which every GPU that loads the library holds until the
 * process exits.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress, with that device current): make that first
 * call before any stream capture.  All calls share the array and it keeps the
 * last call's contents; each call clears what must start at zero on its own
 * stream, and calls that overlap on the GPU (unordered streams) race on it.
 * Non-finite rows, and rows too far from the box to be wrapped, go to cell
 * 0 at the origin as in usr_eval but are not reported.
 * Cost: each cell is sorted by counting, quadratic in its occupancy, so cell
 * edges should be about the cutoff (tens to hundreds of atoms per cell); a
 * mean occupancy above 2,048 atoms per cell is refused.
 * USR_ERR_CAPACITY beyond the limits above (every factor of cells is checked
 * on its own, so no product overflows), USR_ERR_ARG for bad pointers or
 * sizes.  Enqueued on `stream`; no host synchronisation.  n = 0 writes
 * cell_start as all zeros.
 */
usr_status usr_cells_static(int n, const float* xyzq, const double* box, const int* cells, int* cell, int* perm,
                            int* cell_start, float* xw, void* stream);

/*
 * Virial tensor of the last usr_eval of a context created with virial = 1:
 * W = -dE/d(strain) for an affine strain of the box and all positions,
 * row-major 3 x 3 doubles (symmetric), W = W_near + W_far:
 *   W_near = 1/2 sum_{i != j, images, r < r_c} d (x) f_ij    (pair forces of Eq. 20)
 *   W_far_ab = delta_ab E_far - (1/2V) sum_{k != 0} |S(k)|^2 k_a k_b sum_j s_j^2 Fhat_j(k)
 * (the strain derivative of the far energy of Eqs. 4, 9 and F1; the self term of Eq. 10 has
 * none).  The far part is evaluated on the grid: every strain derivative of a Gaussian stays
 * separable (Eq. 31), so W_far_ab - delta_ab E_far = 1/2 <rho, psi_ab> with psi_ab the
 * convolution of rho with s_j^2 d_a d_b of each term's deconvolved kernel.  W is written to
 * `W` (device or host memory, 9 doubles) on `stream`; USR_ERR_ARG without virial = 1 or
 * before any evaluation.
 */
usr_status usr_virial(usr_ctx* ctx, double* W, void* stream);

/*
 * Net charge Q = sum_i q_i of the last evaluation of a context, summed on the
 * GPU by the near + far combination (compensated FP32 within a block, FP64
 * across blocks, fixed order).  A diagnostic: the method assumes a neutral
 * system (Sec. II), and the k = 0 term that a non-zero Q would carry is the
 * one Eq. 4 drops, so for Q != 0 the energy is that quadratic form of the
 * charges.  One double is written to `q` (device or host memory) on `stream`,
 * ordered after the evaluations enqueued before it; 0 for n = 0 and before
 * any evaluation.  USR_ERR_ARG for a NULL context or `q`.
 */
usr_status usr_net_charge(usr_ctx* ctx, double* q, void* stream);

/* Keep (on != 0) or stop keeping the near and far parts of each usr_eval. */
usr_status usr_set_keep_parts(usr_ctx* ctx, int on);

/*
 * Test hook of the failure path (the paper has no counterpart).  With on = 1,
 * the next usr_eval of a tensor-core context (TF32X3 or BF16X3) makes its
 * first convolution pass wait on a barrier that nothing completes; the wait is
 * bounded at 1 ms, as every wait of those kernels is bounded, and runs out.
 * Each CTA of the pass then takes the kernel's own abort path: it raises the
 * timeout bit, waits for its copies in flight, frees its tensor memory and
 * returns, so the context stays usable.  That evaluation's results are not
 * valid and usr_last_device_status reports USR_ERR_TIMEOUT; the hook then
 * clears itself, and the next evaluation is a normal one.  USR_ERR_ARG for an
 * FP32 context.  No GPU fault, trap or unbounded wait is involved.
 */
usr_status usr_debug_inject_timeout(usr_ctx* ctx, int on);

/*
 * Near and far parts of the last usr_eval on this context (which must have
 * run with usr_set_keep_parts on; USR_ERR_ARG otherwise), caller order, n
 * rows float4 each (device; either may be NULL):
 *   near: (F_near, phi_near) of Eq. 20;  far: (F_far, phi_far) of the grid
 *   part, phi_far without the self term.
 */
usr_status usr_debug_parts(usr_ctx* ctx, float* near_out, float* far_out, void* stream);

/* ---- timing ------------------------------------------------------------ */

enum { USR_NSTAGES = 7 };  /* bin, near, spread, conv_x, conv_y, conv_z, gather */

/*
 * Record CUDA events in every usr_eval: on = 1 at every stage boundary, on = 2
 * only just before and after the pair kernel (the least disturbance of the
 * evaluation's timing), 0 none.  USR_ERR_ARG for other values.
 */
usr_status usr_set_profiling(usr_ctx* ctx, int on);

/*
 * Milliseconds of each stage of the last profiled usr_eval (synchronises).
 * ms must hold USR_NSTAGES floats; with profiling level 2 only the near stage
 * (index 1) is measured and the others read 0.  The far chain (spread,
 * conv_x/y/z, then the multilevel coarse steps and the far gather, both
 * counted in gather) runs on the context's own high-priority stream,
 * concurrently with the near stage on the caller's stream; gather also counts
 * the near + far combination after the two streams join.  So the stages can
 * add up to more than the evaluation's duration.
 */
usr_status usr_stage_times(usr_ctx* ctx, float* ms);

/*
 * FP32 fused multiply-add throughput of the current device in TFLOP/s,
 * measured with a register-only loop of two-wide FMAs over every SM (CUDA
 * events around one launch after a warm-up launch; synchronises, allocates a
 * small scratch buffer).  The paper has no counterpart: this is the measured
 * peak that the pair kernel's FP32 roofline fraction divides by.
 */
usr_status usr_fp32_peak(double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* USR_H */
