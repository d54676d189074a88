/*
 * mpm.h -- C ABI of the GB300 box-restricted reaction-diffusion solver.
 *
 * The library advances the species fields of a Cellular Potts lattice by one
 * first-order implicit-Euler, first-order finite-volume step of
 *     dC/dt = D lap(C) - S,       S = k C - q                (Eq. 1-4)
 * restricted to a bounding box of the tumour cells plus a margin (Sec. 2.3),
 * solved by restarted GMRES and mapped back onto the pleural mask (Sec. 2.4),
 * of Dolganov et al., arXiv 2505.03067.  All compute runs in the library's
 * CUDA kernels for sm_103a on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Lattice arrays are dense, x fastest: voxel (i,j,k) is at i + Lx*(j + Ly*k).
 *  - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *    the library never frees them.  Buffers of an mpm_subgrid are owned by the
 *    library and live until mpm_subgrid_destroy / mpm_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Kernels are
 *    queued on it; calls that must size buffers from device results (extract)
 *    synchronise that stream.  Asynchronous CUDA errors surface as
 *    MPM_ERR_CUDA at the next call that synchronises.
 *  - No call throws, exits or prints; each returns an mpm_status and, on error,
 *    leaves a message readable with mpm_last_error(ctx).
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_MAX_SPECIES 4
#define MPM_MAX_RESTART 32

typedef enum {
    MPM_OK = 0,
    MPM_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, id outside tables) */
    MPM_ERR_EMPTY = 2,      /* no tumour voxel (cell id > 0): no box; outputs untouched */
    MPM_ERR_NOCONV = 3,     /* maxit reached; the best iterate is kept */
    MPM_ERR_BREAKDOWN = 4,  /* non-finite value or a zero pivot in the least squares */
    MPM_ERR_TIMEOUT = 5,    /* a bounded inter-CTA wait expired; results are invalid */
    MPM_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    MPM_ERR_NOMEM = 7       /* the context's memory cap or the device is exhausted */
} mpm_status;

typedef struct mpm_ctx mpm_ctx;
typedef struct mpm_subgrid mpm_subgrid;
typedef struct mpm_cnn mpm_cnn;       /* the learned warm start's network (see mpm_cnn_create) */

/* Bounding box: lo inclusive, hi exclusive, per axis (x, y, z). */
typedef struct { int32_t lo[3], hi[3]; } mpm_box;

/* The caller's lattice (all device pointers, caller-owned). */
typedef struct {
    int32_t dims[3];                    /* Lx, Ly, Lz; Lx*Ly*Lz < 2^31 */
    const int32_t *cell_id;             /* CPM cell id per voxel, 0 = medium, > 0 = tumour */
    const uint8_t *mask;                /* 1 = pleural space (solved), 0 = outside */
    const double *dfac;                 /* nullable: per-voxel diffusivity factor (D_s * dfac) */
    double *field[MPM_MAX_SPECIES];     /* concentration of each species (FP64) */
} mpm_lattice;

/* Physical parameters of Eq. 1-4 (host struct; the rate tables are device). */
typedef struct {
    int32_t nspecies;                   /* 1..MPM_MAX_SPECIES */
    int32_t ncell;                      /* entries per species in k_cell / q_cell */
    double dt, h;                       /* time step, grid spacing */
    double D[MPM_MAX_SPECIES];          /* diffusivity */
    double mu[MPM_MAX_SPECIES];         /* uniform first-order decay (Eq. 3-4) */
    double c_bc[MPM_MAX_SPECIES];       /* Dirichlet value on box faces */
    const double *k_cell;               /* device [nspecies][ncell]: uptake of cell id */
    const double *q_cell;               /* device [nspecies][ncell]: source of cell id */
    int32_t bc_box;                     /* 0: Dirichlet box faces, 1: zero flux */
} mpm_params;

typedef struct {
    double rtol;            /* stop when ||b - A x||_2 <= max(rtol*||b||_2, atol) (in-mask rows) */
    double atol;
    int32_t restart;        /* GMRES restart length m, 1..MPM_MAX_RESTART */
    int32_t maxit;          /* total Arnoldi steps per species */
    int32_t precision;      /* 0: FP64 throughout; 1: FP32 Krylov inside FP64 refinement */
    double inner_rtol;      /* precision 1: an FP32 inner cycle stops at max(tol/4, inner_rtol*||r||)
                               (e.g. 1e-6; FP32 cannot reduce much below ~1e-7) */
    int32_t x0_given;       /* 1: the subgrid's current iterate is the initial guess
                               (set by mpm_subgrid_import); 0: c^n from the extract */
    int32_t nblocks;        /* 0: automatic; else the persistent grid size (tuning) */
    int32_t reorth;         /* 1: a second classical Gram-Schmidt pass for an Arnoldi step whose
                               ||w|| fell below 0.7 of its norm before orthogonalisation
                               (the Daniel-Gragg-Kaufman-Stewart test; 0 or 1, else MPM_ERR_ARG; the modified
                               Gram-Schmidt of mpm_solve_fgmres_cnn ignores it) */
    int32_t box_every;      /* mpm_step only (Sec. 2.3's box cadence): 0 or 1, a new bounding box,
                               tile set and neighbour table every step; K > 1, a full extraction
                               on the first step and then every K steps, the steps in between
                               keeping the box and tiles and re-gathering c^n, cell ids and rows.
                               The mask must not change between full extractions. */
    int32_t box_guard;      /* mpm_step with box_every > 1: a tumour voxel (cell id > 0) within
                               box_guard voxels of a box face that is not a lattice face makes
                               the next step a full extraction (0: off).  Negative: MPM_ERR_ARG */
} mpm_opts;

typedef struct {
    int32_t iters[MPM_MAX_SPECIES];     /* Arnoldi steps */
    int32_t cycles[MPM_MAX_SPECIES];    /* restarts (refinement steps for precision 1) */
    int32_t status[MPM_MAX_SPECIES];    /* mpm_status per species */
    int32_t jsum[MPM_MAX_SPECIES];      /* sum over Arnoldi steps of their index j in the cycle */
    double res[MPM_MAX_SPECIES];        /* final true residual ||b - A x||_2 (FP64) */
    double bnorm[MPM_MAX_SPECIES];      /* ||b||_2 over in-mask rows */
    int64_t box_voxels;                 /* nx*ny*nz */
    int64_t mask_voxels;                /* in-mask voxels of the box (the unknowns) */
    int64_t stored_voxels;              /* voxels of the active tiles held in HBM */
    double solve_ms;                    /* device time of the solve kernel (CUDA events; for
                                           mpm_batch_step: of the whole step) */
    double item_ms[MPM_MAX_SPECIES];    /* device time of each species' work item inside the
                                           persistent launch */
    int32_t reorth[MPM_MAX_SPECIES];    /* Arnoldi steps that took the second Gram-Schmidt pass */
    int32_t fallback[MPM_MAX_SPECIES];  /* mpm_solve_fgmres_cnn: 1 when a cycle preconditioned by the
                                           network failed to reduce the FP64 true residual and the
                                           solve went on as plain GMRES (0 elsewhere) */
} mpm_report;

/* Shape of an extracted subgrid (host struct filled by mpm_subgrid_info). */
typedef struct {
    mpm_box box;
    int32_t n[3];               /* box dims */
    int32_t tile[3];            /* tile dims (powers of two) */
    int32_t ntiles;             /* tiles covering the box */
    int32_t nactive;            /* tiles holding at least one in-mask voxel */
    int64_t stored_voxels;      /* nactive * tile volume */
    int64_t mask_voxels;
    int32_t nspecies;
} mpm_subgrid_desc;

/* What mpm_subgrid_export copies out (box-dense layout, x fastest). */
typedef enum {
    MPM_EXPORT_X = 0,       /* current iterate / solution (double), c^n right after extract */
    MPM_EXPORT_RHS = 1,     /* b (double) */
    MPM_EXPORT_DIAG = 2,    /* A_PP (double) */
    MPM_EXPORT_FLAGS = 3,   /* uint8: bits 0-5 open faces -x,+x,-y,+y,-z,+z; bit 6 in mask */
    MPM_EXPORT_CELL = 4     /* int32 cell id */
} mpm_export_what;

/* Create a context on the current CUDA device.  workspace_bytes caps the device
 * memory the library may allocate for subgrids and Krylov bases (0 = no cap).
 * Errors: MPM_ERR_ARG (ctx NULL), MPM_ERR_CUDA (no device). */
mpm_status mpm_create(mpm_ctx **ctx, size_t workspace_bytes);
mpm_status mpm_destroy(mpm_ctx *ctx);
/* Message of the last error on this context ("" if none); valid until the next call. */
const char *mpm_last_error(const mpm_ctx *ctx);

mpm_status mpm_subgrid_create(mpm_ctx *ctx, mpm_subgrid **sub);
mpm_status mpm_subgrid_destroy(mpm_ctx *ctx, mpm_subgrid *sub);
mpm_status mpm_subgrid_info(const mpm_subgrid *sub, mpm_subgrid_desc *out);

/*
 * Sec. 2.3 (dynamic bounding box) + the gather: reduce the lattice to the box
 * of all voxels with cell_id > 0, widened by `margin` and clamped,
 *     lo = max(0, min - margin),  hi = min(L, max + margin + 1),
 * split the box into tiles of dims `tile` (powers of two, product 32..1024;
 * NULL = 4x4x4), keep the tiles that hold an in-mask voxel, and copy the mask,
 * cell ids, optional dfac and the species fields c^n of those tiles into `sub`
 * (tile-major, library-owned).  `nspecies` fields are gathered.
 * Writes the box to *out_box.  Synchronises `stream` once (the compacted
 * size sizes the buffers).  MPM_ERR_EMPTY if no voxel has cell_id > 0:
 * out_box is then unchanged and sub keeps its previous extraction (unless
 * the lattice grew, which invalidates it).
 */
mpm_status mpm_box_extract(mpm_ctx *ctx, const mpm_lattice *lat, int32_t nspecies, int32_t margin,
                           const int32_t tile[3], mpm_box *out_box, mpm_subgrid *sub, void *stream);

/*
 * Refresh a subgrid from the lattice without recomputing its box: re-gather
 * the face flags, cell ids, dfac and the fields c^n of the stored tiles of the
 * last extraction (Sec. 2.3 refreshes the box only every 50 MCS; between
 * refreshes only the fields and cell states change).  The lattice must have
 * the dims of that extraction.  Tiles that gained an in-mask voxel since then
 * are not picked up: call mpm_box_extract again when the mask changes.
 * Invalidates the assembly.  Queued on `stream`, no synchronisation.
 */
mpm_status mpm_subgrid_refresh(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, void *stream);

/*
 * Assemble the implicit-Euler FV system of every species on the extracted box
 * (Eq. 1-4 discretised as in Sec. 2.4).  For an in-mask voxel P:
 *   A_PP = 1 + dt (mu + k_cell[id]) + (dt/h^2) sum_f w_f D_f
 *   A_PQ = -(dt/h^2) D_f   for each face to an in-mask neighbour Q in the box
 *   b_P  = c^n_P + dt q_cell[id] + (dt/h^2) sum_{box faces} 2 D_P c_bc
 * with D_f the harmonic mean of D_s*dfac at P and Q, w_f = 1 on an open face,
 * 2 on a Dirichlet box face (half-cell distance; 0 if bc_box = 1), 0 on a face
 * to a masked voxel.  Masked voxels are identity rows keeping c^n.
 * Queued on `stream`.  MPM_ERR_ARG on bad parameters; a cell id outside
 * [0, ncell) is reported by the next solve as MPM_ERR_ARG.
 */
mpm_status mpm_assemble_coeffs(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_params *prm, void *stream);

/*
 * Solve A c^{n+1} = b for every species of `sub` with restarted GMRES in one
 * persistent kernel (all species in lock step), starting from c^n (or the
 * imported guess), stopping on the true FP64 residual.  precision 1 runs the
 * Krylov basis and operator in FP32 inside FP64 iterative refinement.  If
 * scatter_to is not NULL, the in-mask box voxels of its fields receive the
 * solution (Sec. 2.4); other voxels are untouched.  Synchronises `stream`
 * and fills *rep (may be NULL).  Returns the worst species status.
 */
mpm_status mpm_solve_step(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *scatter_to,
                          const mpm_opts *opt, mpm_report *rep, void *stream);

/*
 * Solve nsys independent subgrids (every species of each) in ONE persistent
 * launch: the grid is split into teams of CTAs; a team takes either one large
 * (system, species) pair on several CTAs or several small ones in turn on one
 * CTA, planned to minimise the longest team's estimated time (per pass a fixed
 * synchronisation cost plus the stored elements over the team's CTAs; the
 * paper's load-imbalance concern, Sec. 2.5).  scatter_to may
 * be NULL or hold nsys entries (each nullable).  reps may be NULL or hold nsys.
 */
mpm_status mpm_solve_batch(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *scatter_to,
                           int32_t nsys, const mpm_opts *opt, mpm_report *reps, void *stream);

/*
 * One implicit-Euler step of nsys extracted systems with fixed boxes (the
 * batched form): for every system refresh c^n from lats[i] (as
 * mpm_subgrid_refresh) and assemble with prms[i], all systems in one launch;
 * then solve every (system, species) pair in ONE persistent launch (as
 * mpm_solve_batch) and scatter the solutions onto lats[i], again one launch.
 * Systems that share a lattice must have disjoint boxes: the scatters of all
 * systems run concurrently.  The first call captures the whole sequence in a
 * CUDA graph; later calls with the same subgrids (not re-extracted), lattice
 * and parameter structs and options replay it (one graph launch per step).
 * Where capture is unavailable the same sequence runs eagerly.  Synchronises
 * `stream` and fills reps (may be NULL; nsys entries).
 */
mpm_status mpm_batch_step(mpm_ctx *ctx, mpm_subgrid *const *subs, const mpm_lattice *const *lats,
                          const mpm_params *const *prms, int32_t nsys, const mpm_opts *opt, mpm_report *reps,
                          void *stream);

/*
 * One implicit-Euler step of every species on a lattice, device-resident:
 * the whole path of Sec. 2.3-2.4 with Eq. 1-4 solved by restarted GMRES --
 * bounding box of the tumour voxels grown by `margin`, tile compaction, the
 * gather of c^n, mask and cell ids with the assembly, the persistent solve
 * and the scatter onto the pleural mask -- with no host round trip between
 * the stages.  The subgrid's buffers are sized for the whole lattice (every
 * box fits), so the box and the element count pass from kernel to kernel in
 * device memory; the host learns them, with the report, once the step is
 * done.  The first call, and any call whose lattice or parameter struct,
 * options, margin or tile differ, captures the stages in a CUDA graph;
 * later calls replay it (one graph launch and one synchronisation of
 * `stream` per step).  The solver grid follows the previous step's element
 * count (re-planned when it moves by more than 25%).
 *   sub     : a subgrid of ctx; after the call it holds this step's extraction
 *             (exports, mpm_apply_operator and mpm_solve_step work on it).
 *   tile    : as in mpm_box_extract (NULL: 4x4x4).
 *   opt     : as in mpm_solve_step; x0_given must be 0 (the step starts at c^n).
 *             box_every / box_guard set the box cadence (default: a new box every
 *             step); the kernel itself decides, step by step, whether to extract
 *             or keep the box, so queued steps follow the cadence too.
 *   rep     : nullable; filled as by mpm_solve_step.
 *   out_box : nullable; the box of this step.
 * Returns MPM_ERR_EMPTY (lattice unchanged, no extraction held) when no voxel
 * has cell_id > 0, MPM_ERR_TIMEOUT (lattice unchanged) when a bounded
 * inter-CTA wait expired, otherwise the status of mpm_solve_step.
 * Device memory per subgrid: about (5 + 36 S) bytes per lattice voxel for the
 * element buffers plus (m + 1) S 4 (FP32 Krylov) or 8 (FP64) bytes per voxel
 * for the Krylov bases (S species, m the restart length), padded to tiles.
 */
mpm_status mpm_step(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm, int32_t margin,
                    const int32_t tile[3], const mpm_opts *opt, mpm_report *rep, mpm_box *out_box, void *stream);

/*
 * mpm_step in two halves, so that a caller can queue steps back to back and
 * keep the host's own work off the device's timeline.  mpm_step_enqueue
 * queues one step on `stream` and returns (the first call, or one whose
 * arguments changed, also builds the graph and synchronises `stream` while
 * doing so); it does not wait for the step.  mpm_step_wait synchronises
 * `stream` and reports the LAST step enqueued on `sub` (rep, out_box and the
 * status as mpm_step returns them; MPM_ERR_ARG if none is pending).  The
 * solver grid is re-planned only from results that were waited for.  The
 * caller must not change the lattice between a step's enqueue and its
 * completion except by stream-ordered work on `stream`.
 */
mpm_status mpm_step_enqueue(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_lattice *lat, const mpm_params *prm,
                            int32_t margin, const int32_t tile[3], const mpm_opts *opt, void *stream);
mpm_status mpm_step_wait(mpm_ctx *ctx, mpm_subgrid *sub, mpm_report *rep, mpm_box *out_box, void *stream);

/*
 * The learned form of the device-resident step (the paper has no network):
 * attach a network (mpm_cnn_* below; its image dims must be the lattice's)
 * and every later mpm_step / mpm_step_enqueue / mpm_step_host on `sub` starts
 * its solve from the network's prediction of c^{n+1} instead of c^n -- in
 * the same CUDA graph, between the extraction and the solve, with no host
 * round trip: features of the step's box, the network on the box's masked
 * voxels, the prediction into the iterate (c^n where it is not finite).  The
 * solve and its stopping rule are unchanged: GMRES corrects the guess.  cnn =
 * NULL detaches.  The network must outlive its use; the graph keeps its
 * buffers.  MPM_ERR_ARG while a step is pending; dims are checked at the
 * next step.
 */
mpm_status mpm_step_set_network(mpm_ctx *ctx, mpm_subgrid *sub, mpm_cnn *cnn);

/* The inputs of a step in host memory, for mpm_step_host (page-locked memory
 * lets the copies run at the link's full speed; pageable memory also works). */
typedef struct {
    const int32_t *cell_id;             /* nullable: the device lattice's cell ids are current */
    const uint8_t *mask;                /* nullable: the device mask is current */
    double *field[MPM_MAX_SPECIES];     /* nullable per species: read with MPM_HOST_FIELDS_IN;
                                           receives the voxels the step updated */
} mpm_host_lattice;

#define MPM_HOST_FIELDS_IN 1            /* mpm_step_host: copy the host fields in before the step */

/*
 * mpm_step with the step's inputs and results in host memory.  On `stream`:
 * copies host->cell_id and host->mask (when not NULL) and, with
 * MPM_HOST_FIELDS_IN, every non-NULL host field into the device lattice `dev`
 * (whose buffers the call overwrites), runs mpm_step on `dev`, waits for it,
 * and copies the voxels the step updated back into the host field of the
 * same species: a page-locked host field (one the device can address)
 * receives the in-mask voxels of the step's box, written by a kernel; any
 * other host field the whole box (one 3-D copy per species, box rows only).
 * A step changes no voxel outside its box nor outside the mask, so a host
 * field that equalled the device field before the step equals it
 * afterwards: a caller that keeps the fields in step (MPM_HOST_FIELDS_IN on
 * the first call and after changing them on the host) moves the cell ids in
 * and the step's results out per step.  The fields are
 * copied back for every status that lets the step write them (MPM_OK,
 * MPM_ERR_NOCONV, MPM_ERR_BREAKDOWN) and left alone otherwise.
 *   dev   : device lattice (as for mpm_step), dims give the size of every copy.
 *   flags : 0 or MPM_HOST_FIELDS_IN; other bits: MPM_ERR_ARG.
 * Other arguments, the return value and the report are those of mpm_step.
 * Synchronous: `stream` is idle when the call returns.
 */
mpm_status mpm_step_host(mpm_ctx *ctx, mpm_subgrid *sub, const mpm_host_lattice *host, const mpm_lattice *dev,
                         const mpm_params *prm, int32_t margin, const int32_t tile[3], const mpm_opts *opt,
                         int32_t flags, mpm_report *rep, mpm_box *out_box, void *stream);

/*
 * Autotuner, tile shape: among the candidate shapes 8x4x4, 8x8x4, 4x4x4,
 * 8x4x2, 16x4x2, 8x8x2, 4x4x2, 16x4x4 pick the one whose active tiles store
 * the fewest voxels for this lattice's box (ties: the larger tile), counted
 * exactly on the device.  Writes the tile to out_tile and the stored-voxel
 * count to *out_stored (nullable).  Synchronises `stream` once per candidate.
 */
mpm_status mpm_tune_tile(mpm_ctx *ctx, const mpm_lattice *lat, int32_t margin, int32_t out_tile[3],
                         int64_t *out_stored, void *stream);

/*
 * Autotuner, restart length and solver kernel variant for a batch of
 * assembled subgrids: times a warm-up and a measured solve from c^n for every
 * candidate (m in {4, 8, 16}; for FP32 with m <= 8 the 4 kernel variants) and
 * keeps the fastest that converges.  Writes m into opt->restart and the
 * variant to *out_variant, and makes that variant the context's default.
 * cache_path (nullable) is a text file of earlier results, keyed by the GPU,
 * precision, tolerance and every system's bucketed box shape and mask
 * occupancy; a hit skips the timing, a miss appends a line.  The iterates are
 * left at c^n.
 */
mpm_status mpm_tune_solver(mpm_ctx *ctx, mpm_subgrid *const *subs, int32_t nsys, mpm_opts *opt,
                           int32_t *out_variant, const char *cache_path, void *stream);

/*
 * Team planner model of the batched solve (the load imbalance of Sec. 2.5):
 * the persistent launch splits its CTAs into teams, and an item (one species
 * of one system) is planned to cost it (F1 + NE) element-equivalents on a
 * one-CTA team and it (F + NE / c) on a team of c > 1 CTAs, it its Arnoldi
 * steps and NE its stored elements.  Each round solves the batch from c^n,
 * fits F1 and F to the measured item times (least squares of the time per
 * Arnoldi step against NE / c, one intercept per regime, every round pooled),
 * takes every item's Arnoldi steps from the solve just measured, and plans
 * again; the round with the smallest imbalance f = t_max / <t> over the teams
 * minus 1 is kept as the context's model (round 0: the unmeasured model;
 * rounds 1..64; it stops early once f has not fallen for two rounds).  Later
 * solves and captured batch steps of a batch with the same item count plan
 * with it.  history (nullable, 3 (rounds + 1) doubles) gets f, F1 and F per
 * round (-1 for rounds not run), out_fixed (nullable, 2 doubles) the kept F1
 * and F.  cache_path as mpm_tune_solver (a hit restores the model; a miss
 * appends F1, F, f, the per-item steps and the per-team times).  The
 * iterates are left at c^n.
 */
mpm_status mpm_tune_teams(mpm_ctx *ctx, mpm_subgrid *const *subs, int32_t nsys, const mpm_opts *opt,
                          int32_t rounds, const char *cache_path, double *history, double *out_fixed,
                          void *stream);

/*
 * Learned warm start (a small 3D CNN; the paper has no network).  Six 3x3x3
 * convolutions with zero padding and biases, channels 9 -> 24 -> 24 -> 24 ->
 * 24 -> 24 -> 3, erf-GELU after layers 1-5, output pred = c^n + s_out * z6
 * (the next-step fields of 3 species), with an activity mask: the network
 * sees the pleural space of its box only (the layer-1 input and activations
 * 1-5 are zero outside the mask or the box, as masked voxels carry no flux,
 * Sec. 2.4).  bf16 weights and activations, FP32 accumulation on the
 * tensor cores (tcgen05); the FP32 master parameters are flat, per layer
 * W[27][Ci][Co] (tap (dx+1) + 3(dy+1) + 9(dz+1)) followed by b[Co].
 * Features (9 channels): c^n of the 3 species (scaled 1, 1, 20), one-hot
 * medium/tumour, per-cell rates (uptake of species 0 and 1, source of
 * species 2; scaled 10), mask.
 *
 * A network works on up to max_images IMAGES of dims image_dims -- lattices
 * of those dims -- each restricted to a box.  Its buffers are indexed like
 * the lattice, so a network whose image dims are a lattice's dims applies to
 * that lattice in place (mpm_cnn_guess, the learned mpm_step).  Device
 * memory: about 82 bytes per image voxel for inference, 500 for training.
 */
#define MPM_CNN_INPUT 0     /* mpm_cnn_load_image: features of the lattice's fields (c^n) */
#define MPM_CNN_TARGET 1    /* mpm_cnn_load_image: the lattice's fields as the training target */
/* train: 0 inference only, 1 also training (keeps activations, gradients, Adam state).
 * Errors: MPM_ERR_ARG (bad dims, max_images outside 1..16, more than 2^31 voxels), MPM_ERR_NOMEM. */
mpm_status mpm_cnn_create(mpm_ctx *ctx, mpm_cnn **cnn, const int32_t image_dims[3], int32_t max_images,
                          int32_t train);
mpm_status mpm_cnn_destroy(mpm_ctx *ctx, mpm_cnn *cnn);
/* Host FP32 parameters (n must equal the network's count); resets Adam; synchronises `stream`. */
mpm_status mpm_cnn_set_params(mpm_ctx *ctx, mpm_cnn *cnn, const float *host_params, int64_t n, float s_out,
                              void *stream);
/* which 0: parameters, 1: the gradient of the last mpm_cnn_train_step (training networks); to host. */
mpm_status mpm_cnn_get_params(mpm_ctx *ctx, const mpm_cnn *cnn, int32_t which, float *host_out, int64_t n,
                              void *stream);
/* Image b (0 <= b < max_images) from a device lattice of the image dims on `box`:
 * MPM_CNN_INPUT sets the image's box and loads mask, features and c^n;
 * MPM_CNN_TARGET loads the lattice's fields as the target (training networks).
 * Queued on `stream`. */
mpm_status mpm_cnn_load_image(mpm_ctx *ctx, mpm_cnn *cnn, int32_t b, const mpm_lattice *lat, const mpm_params *prm,
                              const mpm_box *box, int32_t what, void *stream);
/* Copy of the loaded features of images 0..nimg-1 (x_bf16: [nimg][voxels][16] bf16, channels as
 * above, 9..14 zero, 15 = 1; zero at voxels outside the mask) and their masks (device, caller-owned;
 * only the voxels of each image's box are defined).  Queued on `stream`. */
mpm_status mpm_cnn_export_features(mpm_ctx *ctx, const mpm_cnn *cnn, int32_t nimg, void *x_bf16, uint8_t *mask,
                                   void *stream);
/* Test hook (training networks): the FP32 pre-activations z of layer `layer` (1..5) of images
 * 0..nimg-1 as the last mpm_cnn_train_step computed them, [nimg][voxels][24] into dst (device);
 * defined at the active voxels. */
mpm_status mpm_cnn_export_preact(mpm_ctx *ctx, const mpm_cnn *cnn, int32_t layer, int32_t nimg, float *dst,
                                 void *stream);
/* The network on images 0..nimg-1: pred (device, nullable) [nimg][voxels of an image][3] FP32 receives
 * the prediction at the active voxels (others untouched).  Queued on `stream`. */
mpm_status mpm_cnn_forward(mpm_ctx *ctx, mpm_cnn *cnn, int32_t nimg, float *pred, void *stream);
/* Forward on images 0..nimg-1, mean squared error against their targets over the active voxels and
 * the 3 species, backward; with apply = 1 one Adam step (lr; beta 0.9, 0.999; eps 1e-8).  *loss_out
 * (nullable) gets the loss (synchronises `stream`).  MPM_ERR_TIMEOUT: a bounded wait in a kernel
 * gave up (the context stays usable). */
mpm_status mpm_cnn_train_step(mpm_ctx *ctx, mpm_cnn *cnn, int32_t nimg, float lr, int32_t apply, double *loss_out,
                              void *stream);
/* Initial guess for a solve: features of sub's box from lat (dims = the network's image dims), the
 * network, and the prediction written into the iterate of every species on the in-mask voxels (then
 * solve with x0_given = 1).  A non-finite prediction leaves c^n.  Queued on `stream`. */
mpm_status mpm_cnn_guess(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                         const mpm_params *prm, void *stream);
/* Test hook: device milliseconds of the six convolution launches of the network's last
 * application recorded with MPM_DEBUG_CNN_LAYER_TIMES on (waits for them).  MPM_ERR_ARG when
 * none was recorded. */
mpm_status mpm_cnn_layer_times(mpm_ctx *ctx, mpm_cnn *cnn, float ms[6]);

/*
 * Solve every species of an assembled subgrid by right-preconditioned
 * flexible GMRES(opt->restart) with the network as the preconditioner: for a
 * Krylov vector v of species s, z = m * net(v / m)[s] on the in-mask voxels
 * (m = max |v|), the network's inputs being v in the field channel of s, the
 * other fields and the source map at zero, and the lattice's cell ids, uptake
 * maps and mask over the box (the homogeneous problem, whose solution operator
 * is A^-1).  Each cycle starts from the FP64 true residual r = b - A x and
 * ends with the FP64 update x + Z y (iterative refinement around one flexible
 * GMRES cycle); opt->precision 1 holds the Krylov vectors, the directions z
 * and the operator in FP32 and ends a cycle when its residual estimate falls
 * to max(tol / 4, opt->inner_rtol * ||r||), precision 0 holds them in FP64
 * and ends it at tol.  Classical Gram-Schmidt in two passes, Givens rotations
 * and the least-squares solve in FP64 on the device: the solve is one CUDA
 * graph (conditional WHILE nodes) and the host waits once, for the report.
 * Fallback: a cycle whose true residual is not below the one it started from
 * (or not finite) is discarded and the rest of the solve is plain GMRES
 * (z = v); rep->fallback[s] = 1 records it, and the status is that of the
 * whole solve (a discarded plain cycle ends it: MPM_ERR_NOCONV unless the
 * tolerance is met).  Stopping rule tol = max(rtol ||b_mask||, atol) on the
 * true residual, statuses as mpm_solve_step; rep->reorth counts every Arnoldi
 * step (both passes are always taken).  x0 is c^n, or the iterate as it
 * stands with opt->x0_given = 1 (for instance after mpm_cnn_guess).
 * scatter_to (nullable) receives the result as in mpm_solve_step.  The
 * lattice dims must be the network's image dims; species 0..2 only.
 * MPM_ERR_TIMEOUT: a bounded wait in a network kernel gave up.
 */
/* The preconditioner of mpm_solve_fgmres_cnn applied to one box-dense FP64
 * vector v of species s (device, nx*ny*nz): z (device, box-dense) = the
 * network's z on the stored in-mask voxels, 0 elsewhere.  Queued on `stream`. */
mpm_status mpm_cnn_precond(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                           const mpm_params *prm, int32_t s, const double *v, double *z, void *stream);
mpm_status mpm_solve_fgmres_cnn(mpm_ctx *ctx, mpm_cnn *cnn, mpm_subgrid *sub, const mpm_lattice *lat,
                                const mpm_params *prm, const mpm_lattice *scatter_to, const mpm_opts *opt,
                                mpm_report *rep, void *stream);

/*
 * Growth driver (the CPM of Sec. 2.1 with its mitosis Steppable, Sec. 2.4;
 * the paper gives no Hamiltonian, so this is one simple rule coupled to the
 * fields).  One step, on the device, stream-ordered:
 *  1. growth: every medium voxel (id 0) of the mask with k >= 1 tumour
 *     neighbours (6-neighbourhood; off-lattice neighbours are medium) is taken
 *     over with probability p = p_grow * c_O/(K_o2 + c_O) * c_n/(K_nut + c_n)
 *     (c_O, c_n: field[0], field[1] at the voxel; p = 0 where c_O < o2_min) by
 *     the j-th of its tumour neighbours in the order -x, +x, -y, +y, -z, +z;
 *     every voxel reads the lattice as it was before the step;
 *  2. mitosis: every cell of at least v_div voxels divides, in increasing id
 *     order while the tables have room: the daughter takes id *ncell_dev (then
 *     incremented), the parent's rates (k_cell, q_cell entries written), and
 *     the parent's voxels strictly above its centroid along an axis drawn per
 *     cell (integer test coord * volume > sum of coords).
 * Random numbers: SplitMix64's output function of seed + (c + 1) *
 * 0x9E3779B97F4A7C15, c = ((4 step + stream) mod 2^24) << 40 | index; growth
 * u = (word >> 11) * 2^-53 < p (stream 0, voxel index), neighbour j =
 * ((word >> 32) * k) >> 32 (stream 1), axis = ((word >> 32) * 3) >> 32
 * (stream 2, cell id): the result does not depend on the launch shape.
 * lat: device lattice (cell ids updated in place; mask, field[0], field[1]
 * read).  prm: its rate tables (device, [nspecies][ncell], ncell = capacity;
 * nspecies >= 2) are written for the daughters.  ncell_dev: device int32, the
 * ids in use (medium included), read and updated.  stats_dev: device int64[3]
 * accumulating grown voxels, divisions, and voxels whose id lies outside
 * [0, capacity) (left unchanged).  MPM_ERR_ARG on a null or inconsistent
 * argument, p_grow, K_o2 or K_nut negative or NaN, v_div < 2, step < 0.
 */
typedef struct {
    double p_grow;      /* growth probability at saturating O2 and nutrient */
    double K_o2;        /* half-saturation concentration of O2 (species 0) */
    double K_nut;       /* half-saturation concentration of the nutrient (species 1) */
    double o2_min;      /* no growth into a voxel whose O2 is below this */
    int32_t v_div;      /* a cell of at least v_div voxels divides */
    int32_t reserved;
} mpm_cpm_params;
mpm_status mpm_cpm_step(mpm_ctx *ctx, const mpm_lattice *lat, const mpm_params *prm, const mpm_cpm_params *cp,
                        uint64_t seed, int64_t step, int32_t *ncell_dev, int64_t *stats_dev, void *stream);

/* Copy `what` of species s from the subgrid into dst (device, box-dense,
 * nx*ny*nz elements of the export type).  Voxels of tiles that hold no
 * in-mask voxel are not stored: they receive 0 (1 for DIAG).  Queued on
 * `stream`. */
mpm_status mpm_subgrid_export(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t what, int32_t s,
                              void *dst, void *stream);

/* Overwrite the iterate of species s with src (device, box-dense doubles) on
 * the in-mask voxels: the initial guess used when opts.x0_given = 1. */
mpm_status mpm_subgrid_import(mpm_ctx *ctx, mpm_subgrid *sub, int32_t s, const double *src, void *stream);

/* y = A x for species s (device, box-dense doubles, FP64 operator of the last
 * assemble): the matrix-free 7-point operator alone. */
mpm_status mpm_apply_operator(mpm_ctx *ctx, const mpm_subgrid *sub, int32_t s, const double *x,
                              double *y, void *stream);

/* Scatter the current iterate to the lattice (in-mask box voxels only). */
mpm_status mpm_scatter(mpm_ctx *ctx, const mpm_subgrid *sub, const mpm_lattice *lat, void *stream);

/* Test hooks for failure detection (no GPU fault is ever provoked):
 *  MPM_DEBUG_TIMEOUT_NS  wall-time limit of every inter-CTA wait of the solver
 *                        (default 2e9 ns); on expiry the solve returns
 *                        MPM_ERR_TIMEOUT and the context stays usable.
 *  MPM_DEBUG_SKIP_BLOCK  CTA index that leaves the solver at once, so that its
 *                        partners' waits run out (-1 = none, the default).
 *  MPM_DEBUG_PHASE_TIMES 1: CTA 0 of every later solve records where its time
 *                        went (read with the MPM_COUNTER_PHASE_* counters).
 *  MPM_DEBUG_SOLVER_VARIANT  solver kernel variant 0..6 (elements in flight per
 *                        thread, CTAs per SM, threads per CTA; 0 = default;
 *                        a bucket without the variant uses its default), for
 *                        tuning.
 *  MPM_DEBUG_CNN_LAYER_TIMES 1: every later network application outside a
 *                        graph capture records CUDA events around each of its
 *                        six convolution launches (read with
 *                        mpm_cnn_layer_times). */
#define MPM_DEBUG_TIMEOUT_NS 1
#define MPM_DEBUG_SKIP_BLOCK 2
#define MPM_DEBUG_PHASE_TIMES 3
#define MPM_DEBUG_SOLVER_VARIANT 4
#define MPM_DEBUG_CNN_LAYER_TIMES 5
mpm_status mpm_debug_set(mpm_ctx *ctx, int32_t key, int64_t value);

/* Test hook: the FP32 Krylov path's bit-level conversions applied to n
 * device values, with CUDA's own conversions beside them as the reference:
 * out32[i] = in64[i] rounded toward zero to FP32 by integer operations
 * (magnitudes below FP32's normal range, 2^-126, give a signed zero where
 * CUDA gives a subnormal; magnitudes of 2^128 and above give infinity where
 * CUDA's round-toward-zero gives the largest finite FP32; NaN stays NaN),
 * ref32[i] = __double2float_rz(in64[i]); out64[i] = in32[i] widened by
 * integer operations (FP32 subnormals give a signed zero), ref64[i] =
 * (double)in32[i].  All device arrays of n entries; queued on `stream`.
 * MPM_ERR_ARG for n < 0 or a null pointer. */
mpm_status mpm_debug_convert(const double *in64, float *out32, float *ref32, const float *in32, double *out64,
                             double *ref64, int64_t n, void *stream);

/* Counters of the context: MPM_COUNTER_LAUNCHES = kernels launched so far by
 * this context (every entry point counts its own launches); with
 * MPM_DEBUG_PHASE_TIMES on, the last solve's CTA-0 nanoseconds spent in the
 * streaming passes (WORK), waiting at team barriers (WAIT), summing the team's
 * partial sums (REDUCE) and in the FP64 least-squares/state updates (SERIAL). */
#define MPM_COUNTER_LAUNCHES 1
#define MPM_COUNTER_BATCH_GRAPH 10   /* 1 if the last mpm_batch_step replays a captured graph */
/* Load imbalance of the last solve, the paper's f = t_max / <t> - 1 (Sec. 2.5)
 * with the CTA teams of the persistent launch in place of the cores, in parts
 * per million. */
#define MPM_COUNTER_IMBALANCE_PPM 11
#define MPM_COUNTER_PHASE_WORK_NS 2
#define MPM_COUNTER_PHASE_WAIT_NS 3
#define MPM_COUNTER_PHASE_REDUCE_NS 4
#define MPM_COUNTER_PHASE_SERIAL_NS 5
/* WORK split by pass: residual, Arnoldi pass 1 (matvec + dots), pass 2
 * (orthogonalisation + norm), solution update. */
#define MPM_COUNTER_PHASE_R_NS 6
#define MPM_COUNTER_PHASE_P1_NS 7
#define MPM_COUNTER_PHASE_P2_NS 8
#define MPM_COUNTER_PHASE_U_NS 9
/* mpm_step only: time of the extraction (up to the grid barrier that ends it)
 * and of the wait for the last team plus the scatter, on CTA 0. */
#define MPM_COUNTER_PHASE_EXTRACT_NS 12
#define MPM_COUNTER_PHASE_SCATTER_NS 13
/* mpm_step only, the extraction's phases each up to its grid barrier: the
 * bounding box, the tile activity, the active-tile counts (a phase of its own
 * only for boxes of more than 64 Ki tiles; otherwise counted within the
 * compaction and near 0 here), the compaction and the gather + rows (the last
 * without a barrier). */
#define MPM_COUNTER_PHASE_BBOX_NS 14
#define MPM_COUNTER_PHASE_ACTIVITY_NS 15
#define MPM_COUNTER_PHASE_COUNT_NS 16
#define MPM_COUNTER_PHASE_COMPACT_NS 17
#define MPM_COUNTER_PHASE_GATHER_NS 18
/* mpm_step: full extractions (new box, tile set and neighbour table) since the
 * step's graph was last set up, as of the last step waited for (with
 * mpm_opts.box_every > 1 the other steps keep the box). */
#define MPM_COUNTER_STEP_FULL_EXTRACTIONS 19
mpm_status mpm_counter_get(const mpm_ctx *ctx, int32_t key, int64_t *value);

/*
 * Bounding box without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, for
 * example code whose device memory is all owned by another allocator (a
 * framework's caching allocator or a pool fixed at start-up), code that must
 * not risk the device-wide synchronisation that cudaMalloc/cudaFree can
 * cause, or a plugin whose host application controls every allocation.  It
 * needs no context (creating one allocates) and calls no allocating routine.
 *
 * Computes the same box as mpm_box_extract (voxels with cell_id > 0, widened
 * by `margin`, clamped to the lattice) and writes to out_box (device memory,
 * 7 int32, caller-owned): lo[3], hi[3] (exclusive) and a found flag (0 when
 * no voxel has cell_id > 0; lo and hi are then 0).  cell_id is the caller's
 * device lattice of dims Lx*Ly*Lz < 2^31.  Kernels are queued on `stream`
 * (cudaStream_t, NULL = legacy default); nothing synchronises.
 *
 * Scratch: one fixed array of MPM_NOALLOC_MAX_SLABS * 8 int32 (128 KB) per
 * partial bound of each z-slice, compiled into the library; every GPU that
 * loads the library holds it until the process exits.  All calls share it
 * and each call overwrites what it reads, so calls that overlap on the GPU
 * (on different streams or different host threads) race.  The first call on
 * a device looks up the array's device address with that device current
 * and keeps it; make that first call before any stream capture.  The address
 * is not looked up again: after cudaDeviceReset on a device, do not call
 * this entry point on that device in the same process.
 *
 * Errors: MPM_ERR_ARG (null pointer, negative margin, bad dims),
 * MPM_ERR_NOMEM (Lz > MPM_NOALLOC_MAX_SLABS: more z-slices than the fixed
 * scratch holds), MPM_ERR_CUDA (symbol lookup or launch failed).
 */
#define MPM_NOALLOC_MAX_SLABS 4096
mpm_status mpm_box_bounds_noalloc(const int32_t *cell_id, const int32_t dims[3], int32_t margin, int32_t *out_box,
                                  void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MPM_H */
