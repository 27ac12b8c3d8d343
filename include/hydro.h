/*
 * hydro.h -- C ABI of the GB300 (sm_103a) hydro library: one second-order unsplit
 * MUSCL-Hancock step (PLM primitive reconstruction, Hancock half-step predictor, HLLC fluxes,
 * conservative update) of the 3D ideal-gas Euler equations on AMR grid patches, the per-patch
 * CFL time step, Ramses-style oct groups (gathered, read in place, or through a device-built
 * Morton order and neighbour table), the adjoint of the step, the coupling of AMR levels
 * (coarse-fine ghosts, flux registers, refluxing, average-down), a PPM variant, and ideal MHD
 * with hyperbolic divergence cleaning.
 *
 * What the calls compute follows the paper's description of the hydro path: the baryonic
 * component is an ideal fluid governed by the Euler equations, solved with PLM among other
 * methods (Sec. 2); the GPU computes every flux that updates a patch's cells, with an adaptive
 * time step (Sec. 4, Enzo); hydro solved on chunks of patches that carry their
 * boundary cells (Sec. 3, Ramses GPU procedure); the N_v x 6^3 gathered cell buffer (Sec. 3).
 * The paper prints no equations; the scheme is the textbook one, with these readings: primitive
 * reconstruction; MinMod / MC / unlimited slopes; unsplit primitive Hancock predictor summed over
 * x, y, z; Davis wave speeds and Batten et al. star states in HLLC; dt = cfl * dx /
 * max(|u|+|v|+|w|+3c); density and pressure floors after recovery and on face states.
 *
 * Conventions
 *   - Every field pointer is DEVICE memory owned by the caller; the library never frees it.
 *     Fields are structure-of-arrays: five separate arrays (rho, m_x, m_y, m_z, E), x fastest.
 *     Element type: double for HYDRO_FP64, HYDRO_MIXED and HYDRO_FP64_DF, float for HYDRO_FP32.
 *   - The library owns only what a hydro_ctx holds: the device error word, uploaded patch
 *     descriptors, the tile work-list and its counter, captured CUDA graphs, autotune results.
 *   - Every call is asynchronous on the context's stream, except hydro_get_error (and
 *     hydro_autotune), which synchronise it.  After a first call with a given patch set, calls
 *     with the same set allocate nothing and can be captured in a CUDA graph.
 *   - Argument errors are detected on the host and return HYDRO_ERR_ARG before anything is
 *     launched.  Physical errors found on the device set bits of the error word
 *     (HYDRO_EBIT_*), read back by hydro_get_error.  CUDA errors return HYDRO_ERR_CUDA.
 *   - Ghost cells: a patch with ng == 2 carries two ghost layers filled by the caller (the paper's
 *     chunks carry their boundary cells, Sec. 3); three (ng == 3) for the PPM reconstruction.
 *     ng == 0 means a periodic box: the library wraps indices itself.
 */
#ifndef HYDRO_H
#define HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYDRO_OK = 0,
  HYDRO_ERR_ARG = -1,        /* bad argument; nothing launched */
  HYDRO_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  HYDRO_ERR_UNPHYSICAL = -3, /* hydro_get_error: the error word is non-zero */
  HYDRO_ERR_TIMEOUT = -4,    /* a bounded device wait ran out */
  HYDRO_ERR_NOMEM = -5,      /* device allocation of library-owned scratch failed */
  HYDRO_ERR_STATE = -6       /* call not valid in the context's current state */
} hydro_status;

typedef enum { HYDRO_FP64 = 0, HYDRO_FP32 = 1, HYDRO_MIXED = 2, HYDRO_FP64_DF = 3 } hydro_precision;
/* HYDRO_FP64 : double state, double arithmetic throughout.
 * HYDRO_FP32 : float state; float reconstruction, predictor, HLLC and update; the pressure
 *              recovery p = (gamma-1)(E - |m|^2/(2 rho)) is evaluated with error-free float
 *              transformations to double-float accuracy (at least as accurate as evaluating it in
 *              double and rounding to float).
 * HYDRO_MIXED: double state; the pressure recovery to double-float accuracy from the double
 *              state split exactly into float pairs (error-free float transformations, no FP64
 *              arithmetic); float reconstruction, predictor, HLLC and flux divergence; the update
 *              U + dU accumulated in double.
 * HYDRO_FP64_DF: double state; every step of the scheme in double-float arithmetic (pairs of
 *              floats, about 48 significant bits, on the FP32 pipes), the update U + dU accumulated
 *              in double.  Same results as HYDRO_FP64 to about 1e-13 relative, several times faster
 *              on parts whose FP64 rate is a small fraction of their FP32 rate.  Its exponent range
 *              is that of float: the intermediates of the scheme (state, speeds, fluxes, products
 *              such as |m|^2 and rho u^2) keep the FP64 accuracy only between about 1e-30 and 3e38
 *              in magnitude -- below, the low float of a pair leaves the normal range and relative
 *              accuracy drops towards float's (for |m|^2 below ~1e-38, to nothing); above, they
 *              overflow, which the recovery flags as HYDRO_EBIT_NONFINITE. */

typedef enum { HYDRO_MINMOD = 0, HYDRO_MC = 1, HYDRO_NOLIMIT = 2, HYDRO_PPM = 3 } hydro_limiter;
/* HYDRO_MINMOD, HYDRO_MC, HYDRO_NOLIMIT: piecewise-linear (PLM) reconstruction with that slope.
 * HYDRO_PPM:  piecewise-parabolic reconstruction (Colella & Woodward 1984; the paper lists PPM
 *             among its hydro methods, Sec. 2): fourth-order interface values from MC-limited
 *             slopes, the monotonicity constraints on each cell's edges, the Hancock predictor with
 *             the parabola's centre slope and face states q_h + (edge - q).  Stencil radius 3:
 *             hydro_step takes a periodic box (ng == 0) or patches carrying three ghost layers
 *             (ng == 3; ng == 2 patches are refused), and hydro_run a periodic box.  The host-buffer,
 *             oct, flux-register and adjoint calls return HYDRO_ERR_ARG for a PPM context. */

/* Bits of the device error word. */
#define HYDRO_EBIT_NONFINITE 0x01u /* a recovered density or pressure was not finite */
#define HYDRO_EBIT_RHO_FLOOR 0x02u /* recovered density below rho_floor (floored) */
#define HYDRO_EBIT_P_FLOOR 0x04u   /* E below the kinetic energy: negative pressure (floored) */
#define HYDRO_EBIT_BAD_DT 0x08u    /* a step was given dt <= 0 or non-finite (no update done) */
#define HYDRO_EBIT_BAD_TILE 0x10u  /* a work-list record pointed outside its patch */
#define HYDRO_EBIT_TIMEOUT 0x20u   /* a bounded device wait gave up */
#define HYDRO_EBIT_OOB 0x40u       /* bounds-checked build only (HYDRO_CHECK_BOUNDS): a step kernel
                                      computed a global index outside its patch's array; that
                                      access was skipped.  Never set by the default build. */

typedef struct {
  double gamma;      /* ratio of specific heats, > 1 */
  double cfl;        /* Courant number C of the dt formula, in (0, 1] */
  double rho_floor;  /* density floor, >= 0 */
  double p_floor;    /* pressure floor, >= 0 */
  int limiter;       /* hydro_limiter */
  int precision;     /* hydro_precision */
  void* cuda_stream; /* cudaStream_t all calls are enqueued on; NULL = legacy default stream */
} hydro_config;

typedef struct {
  void* U[5];        /* device pointers to rho, m_x, m_y, m_z, E (see the element type above);
                        host pointers for hydro_step_host only */
  int nx, ny, nz;    /* interior cells, each >= 1 */
  int ng;            /* ghost layers: 2 (caller-filled; 3 in a HYDRO_PPM context) or 0 (periodic box,
                        wrapped by the library) */
  long long sy, sz;  /* element strides of y and z in the stored (ghosted) array; x stride is 1.
                        Require sy >= nx + 2 ng and sz >= sy * (ny + 2 ng). */
  double dx;         /* cell size, > 0 */
  int level;         /* refinement level (informational; dx carries the geometry) */
} hydro_patch;

typedef struct hydro_ctx hydro_ctx;

/* Create a context on the current CUDA device (library bookkeeping, no counterpart in the paper;
 * cfg holds the ideal-gas gamma of Sec. 2 and the CFL number of the adaptive step, Sec. 4).
 * Validates cfg (gamma > 1, 0 < cfl <= 1,
 * floors >= 0, enums in range) and allocates the device error word.  *ctx is set to NULL on
 * failure.  Returns HYDRO_OK, HYDRO_ERR_ARG, HYDRO_ERR_NOMEM or HYDRO_ERR_CUDA. */
int hydro_init(hydro_ctx** ctx, const hydro_config* cfg);

/* Synchronise the context's stream and free everything the context owns (no counterpart in the
 * paper).  NULL is a no-op. */
int hydro_finalize(hydro_ctx* ctx);

/* Per-patch CFL time step (adaptive time step, Sec. 2 and Sec. 4):
 *   dt_dev[p] = cfl * dx_p / max over the interior cells of patch p of (|u|+|v|+|w| + 3 c),
 *   c = sqrt(gamma p / rho), from the recovered (floored) primitive state.
 * p: host array of npatch descriptors (npatch >= 1).  dt_dev: device array of npatch doubles,
 * overwritten.  In HYDRO_FP32 and HYDRO_MIXED the per-cell speeds are float; the dt formula is
 * evaluated in double.  The result is bit-identical to the dt_next output of hydro_step on the
 * same state. */
int hydro_cfl_dt(hydro_ctx* ctx, const hydro_patch* p, int npatch, double* dt_dev);

/* One MUSCL-Hancock/HLLC step of every patch (recovery, PLM slopes -- or the PPM parabola in a
 * HYDRO_PPM context --, Hancock predictor, HLLC fluxes on every face, conservative update; Sec. 2
 * and Sec. 4):
 *   out[p] interior <- U^{n+1} of in[p] with time step dt_dev[p] and cell size in[p].dx.
 * in, out: host arrays of npatch descriptors with equal nx, ny, nz and dx per patch; out[p] may
 * have ng 0, 2 or (PPM) 3 (only its interior is written) and must not overlap in[p] (use two buffers).
 * dt_dev: device array of npatch doubles.  dt_next_dev: NULL, or a device array of npatch
 * doubles that receives the CFL dt of U^{n+1} (same formula as hydro_cfl_dt), fused into the
 * step.  A single periodic box (npatch == 1, ng == 0) runs the uniform-grid kernel; any other
 * set (in[p] with ng == 2, or 3 in a HYDRO_PPM context) runs one persistent launch over a
 * device-built tile work-list.  The descriptors are
 * uploaded and the work-list rebuilt only when the patch set differs from the previous call's. */
int hydro_step(hydro_ctx* ctx, const hydro_patch* in, const hydro_patch* out, int npatch, const double* dt_dev,
               double* dt_next_dev);

/* One step of Ramses-style oct groups (Sec. 3: the N_v x 6 x 6 x 6 gathered buffer): each
 * group is the 2x2x2 oct plus two ghost layers, gathered by the caller.
 *   gathered[f]: device array [ngroups][6][6][6] (z, y, x) of field f;
 *   out[f]:      device array [ngroups][2][2][2] receiving U^{n+1} of the oct's 8 cells.
 * All groups share dx and the time step dt_dev[0].  ngroups >= 1. */
int hydro_step_octs(hydro_ctx* ctx, void* const gathered[5], void* const out[5], long long ngroups, double dx,
                    const double* dt_dev);

/* Fill the two ghost layers of fine patches from the next-coarser level (refinement ratio 2), the
 * boundary-cell interpolation of the paper's Ramses chunk builder (Sec. 3): conservative
 * piecewise-linear prolongation of each conserved variable with MinMod-limited slopes,
 *     U_f = U_C + s_x D_x + s_y D_y + s_z D_z,  s_d = +-1/4,  D_d = minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C),
 * for a fine cell with fine-level index f in coarse cell C = floor(f/2) (upper half when f is odd),
 * the coarse level periodic.  The eight children of a coarse cell average to it.
 *   coarse:       the coarse level as a periodic box (ng == 0);
 *   fine:         npatch patches with ng == 2 and dx == coarse->dx / 2; only their ghost cells are
 *                 written, the interiors are left untouched; they must not overlap the coarse
 *                 level or one another;
 *   fine_origins: host array [npatch][3] of int (x, y, z): the fine-level index of each patch's
 *                 first interior cell (any integers: fine indices wrap with the level's period).
 * Arithmetic in the storage type.  A call with a patch set different from the previous call's
 * uploads its descriptors and synchronises the stream first. */
int hydro_fill_ghosts(hydro_ctx* ctx, const hydro_patch* coarse, const hydro_patch* fine, const int* fine_origins,
                      int npatch);

/* The same ghost fill from the coarse level interpolated in time within its step, for a finer level
 * that advances by smaller steps between the coarse ones (time refinement, Sec. 2): each coarse
 * value used is (1 - theta) * coarse_old + theta * coarse_new, each product and the sum rounded once
 * in the storage type, then prolonged as by hydro_fill_ghosts.  coarse_old, coarse_new: the coarse
 * level before and after its step (ng == 0, same sizes and strides); 0 <= theta <= 1 (theta = 1
 * gives hydro_fill_ghosts on coarse_new, theta = 0 on coarse_old, bit for bit). */
int hydro_fill_ghosts_time(hydro_ctx* ctx, const hydro_patch* coarse_old, const hydro_patch* coarse_new, double theta,
                           const hydro_patch* fine, const int* fine_origins, int npatch);

/* Same-level ghost exchange (the boundary cells a chunk carries, Sec. 3, where a neighbouring patch
 * of the same level covers them): every ghost cell of a patch that lies in the interior of a patch of the
 * same level (another one, or the patch itself across the period) takes that interior cell's
 * values; other ghost cells are left as they are (fill them from the coarser level first with
 * hydro_fill_ghosts).  The level is periodic with period[3] = (x, y, z) fine cells.
 *   fine:    npatch patches, ng == 2, interiors no larger than the period and not overlapping one
 *            another (modulo the period); they must not share memory;
 *   origins: host array [npatch][3] of int: each patch's first interior cell (wrapped by the period).
 * Deterministic (each ghost cell has at most one source).  A call with a patch set different from
 * the previous call's builds its copy list on the host (a spatial hash of the interiors) and
 * synchronises the stream first. */
int hydro_exchange_ghosts(hydro_ctx* ctx, const hydro_patch* fine, const int* origins, int npatch, const int period[3]);

/* Flux registers, refluxing and average-down: the coupling of two AMR levels (refinement ratio 2)
 * that keeps the composite level conservative (Berger & Colella 1989; the paper's GPU ports compute
 * every flux that updates a patch's cells, Sec. 4, and the coarse level's fluxes at a fine patch's
 * boundary must then become the fine ones).  A register holds, per field, the time-integrated
 * fluxes dt * F through the six boundary faces of a box of nx x ny x nz cells, in the storage type:
 *     x-low [nz][ny], x-high [nz][ny], y-low [nz][nx], y-high [nz][nx], z-low [ny][nx], z-high [ny][nx]
 * (5 x 2 (ny nz + nx nz + nx ny) elements; device memory owned by the caller).  The fluxes are the
 * ones hydro_step applies there for the same state and dt: recovery, limited slopes and predictor
 * of the two adjacent cells, floored face states, HLLC.
 *   hydro_patch_fluxes: the boxes are the interiors of ghosted patches (ng == 2) with time steps
 *       dt_dev[p]; registers[p] receives dt * F (accumulate == 0) or adds it (accumulate != 0: the
 *       integral over a fine patch's substeps).
 *   hydro_level_fluxes: the boxes (host arrays box_origins, box_dims [nbox][3] of int, x y z;
 *       origins wrapped by the level's size, sizes no larger than it) of a periodic level (ng == 0),
 *       all with time step dt_dev[0].
 *   hydro_reflux: after the coarse step, each coarse cell outside box b across one of its faces gets
 *       s/dx (Rc - mean of the four fine faces' Rf), s = +1 below the box, -1 above; Rc =
 *       coarse_registers[b] (the box's coarse register), Rf = fine_registers[b] (the register of
 *       the fine patch covering it, box sizes doubled).  Boxes must not overlap; the six face kinds
 *       are applied in turn, so the result is deterministic.
 *   hydro_average_down: the coarse cells under each fine patch's interior (fine origin and sizes
 *       even) become the mean of their eight children.
 * A call whose descriptors differ from the previous call of the same kind uploads them and
 * synchronises the stream first. */
int hydro_patch_fluxes(hydro_ctx* ctx, const hydro_patch* patches, int npatch, const double* dt_dev,
                       void* const* registers, int accumulate);
int hydro_level_fluxes(hydro_ctx* ctx, const hydro_patch* level, const int* box_origins, const int* box_dims, int nbox,
                       const double* dt_dev, void* const* registers, int accumulate);
int hydro_reflux(hydro_ctx* ctx, const hydro_patch* coarse, const int* box_origins, const int* box_dims, int nbox,
                 void* const* coarse_registers, void* const* fine_registers);
int hydro_average_down(hydro_ctx* ctx, const hydro_patch* coarse, const hydro_patch* fine, const int* fine_origins,
                       int npatch);

/* Oct groups read in place from a periodic level grid instead of a gathered buffer (the paper's
 * Ramses GPU procedure gathers each oct's neighbourhood into an N_v x 6^3 buffer first, Sec. 3;
 * here each group's 6^3 stencil is read from the level with periodic wrap as it is needed).
 *   level:       a periodic box (ng == 0, each of nx, ny, nz >= 4) of the level's cells; dx is
 *                the level's cell size;
 *   origins_dev: device array [ngroups][3] of int (x, y, z): the oct's lowest cell, in [0, n)
 *                per axis (an origin outside the grid sets HYDRO_EBIT_BAD_TILE and that group's
 *                output is left unwritten);
 *   out[f]:      device array [ngroups][2][2][2] (z, y, x) receiving U^{n+1} of the oct's cells.
 * Same arithmetic, so the same bits, as hydro_step_octs on the gathered stencils. */
int hydro_step_octs_level(hydro_ctx* ctx, const hydro_patch* level, const int* origins_dev, long long ngroups,
                          void* const out[5], const double* dt_dev);

/* The device chunk builder's bookkeeping for one level's octs (Sec. 3 and Fig. 1: the Ramses GPU
 * procedure orders a level's cells along the space-filling curve and gathers each oct's
 * neighbourhood for the hydro kernel).  An oct at oct coordinates (X, Y, Z) holds the level's cells
 * 2X..2X+1, 2Y..2Y+1, 2Z..2Z+1; the level is periodic with dims[3] = (X, Y, Z) octs per axis.
 *
 * hydro_octs_build: the Morton order of the octs and their neighbour table.
 *   pos_dev:   device array [noct][3] of int, oct coordinates (X, Y, Z), each in [0, dims);
 *   dims:      host array of 3 ints, each in 1..1024; 1 <= noct <= 2^28;
 *   order_dev: device array [noct] of int, receives the oct indices in increasing Morton key
 *              (bits of X, Y, Z interleaved, x lowest);
 *   nbr_dev:   NULL, or a device array [noct][27] of int that receives, in entry
 *              ((dz+1)*3 + dy+1)*3 + dx+1 of oct o, the index of the oct at (X+dx, Y+dy, Z+dz)
 *              wrapped on the level, or -1 where the level has no oct; entry 13 is o.
 *   A position outside dims, or two octs at one position, sets HYDRO_EBIT_BAD_TILE; order and the
 *   table are then not meaningful (order entries left without an oct are -1).  The scratch (a
 *   bitmap over 8^b keys, 2^b >= max dims) is owned by the context and grows on demand.
 *
 * hydro_step_octs_table: one step of the octs list_dev[0 .. ngroups-1] of an oct-major level whose
 * 6^3 stencils are read through the neighbour table (stencil cell (x, y, z), each 0..5, is cell
 * (x%2, y%2, z%2) of the neighbour at offset (x/2 - 1, y/2 - 1, z/2 - 1)).
 *   in[f], out[f]: device arrays [noct][2][2][2] (cell (i, j, k) of oct o at o*8 + (k*2 + j)*2 + i),
 *              in and out not overlapping; the listed octs' cells in out receive U^{n+1}, the other
 *              octs' cells are left as they are;
 *   nbr_dev:   the table of hydro_octs_build (or the caller's, same layout);
 *   list_dev:  device array [ngroups] of oct indices (e.g. order_dev, or a part of it).
 *   A listed oct outside [0, noct), or one with a neighbour entry outside it (-1 included: every
 *   listed oct needs its 26 neighbours), sets HYDRO_EBIT_BAD_TILE and is skipped.
 *   All octs share dx and dt_dev[0].  Same arithmetic, so the same bits, as hydro_step_octs on the
 *   gathered stencils. */
int hydro_octs_build(hydro_ctx* ctx, const int* pos_dev, int noct, const int dims[3], int* order_dev, int* nbr_dev);
int hydro_step_octs_table(hydro_ctx* ctx, void* const in[5], void* const out[5], int noct, const int* nbr_dev,
                          const int* list_dev, long long ngroups, double dx, const double* dt_dev);

/* Ideal magnetohydrodynamics on a periodic box, the second workload (the paper's Enzo runs MHD on
 * the GPU, Sec. 4; it prints no equations).  Nine fields, each a device array of nx*ny*nz elements,
 * x fastest: rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi, with E = p/(gamma-1) + |m|^2/(2 rho) +
 * |B|^2/2 (magnetic pressure |B|^2/2) and psi the scalar of hyperbolic divergence cleaning
 * (Dedner et al. 2002).  One step: primitive variables (rho, u, v, w, p, B, psi) reconstructed
 * with the context's PLM limiter; conservative unsplit Hancock predictor (each extrapolated state
 * minus dt/(2 dx) times the sum over axes of the flux differences of the cell's own extrapolated
 * states), recovered and floored; HLL fluxes with Davis bounds from the fast magnetosonic speed,
 * the normal field and psi at each face from the 2x2 cleaning system with c_h = (cfl/3) dx/dt;
 * conservative update; psi scaled by exp(-0.4 c_h dt/dx).
 *   hydro_mhd_step: out <- U^{n+1} of in with time step dt_dev[0]; in and out must not overlap;
 *       dt_next_dev: NULL or one double receiving cfl dx / max_cells sum_d (|u_d| + c_f,d) of U^{n+1}.
 *       HYDRO_FP32 and HYDRO_MIXED run one fused launch with no per-cell scratch; HYDRO_FP64 and
 *       HYDRO_FP64_DF use 81 elements per cell of device scratch (face states and fluxes), owned
 *       by the context.
 *   hydro_mhd_cfl_dt: dt_dev[0] <- the same CFL dt of U (bit-identical to the fused one).
 * Element type: double in HYDRO_FP64, HYDRO_FP64_DF (double-float arithmetic, the update summed in
 * double) and HYDRO_MIXED (the state read as float, float arithmetic, the update summed in double)
 * contexts, float in HYDRO_FP32; a HYDRO_PPM context returns HYDRO_ERR_ARG, as do sizes with
 * nx*ny*nz >= 2^31.  Floors and error bits as the hydro step. */
int hydro_mhd_step(hydro_ctx* ctx, void* const in[9], void* const out[9], int nx, int ny, int nz, double dx,
                   const double* dt_dev, double* dt_next_dev);
int hydro_mhd_cfl_dt(hydro_ctx* ctx, void* const U[9], int nx, int ny, int nz, double dx, double* dt_dev);

/* The same MHD step on AMR patches that carry two ghost layers filled by the caller (the paper's
 * chunks carry their boundary cells, Sec. 3), many patches per call (one launch per stage over a
 * block table of all patches).  A patch: */
typedef struct {
  void* U[9];        /* device pointers: rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi */
  int nx, ny, nz;    /* interior cells */
  int ng;            /* ghost layers: 2 (inputs and the CFL), 0 or 2 (outputs: only the interior is written) */
  long long sy, sz;  /* element strides of y and z in the stored array; x stride 1 */
  double dx;         /* cell size, > 0 */
  int level;         /* refinement level (informational) */
} hydro_mhd_patch;
/* MHD on patches (Sec. 4, Enzo's MHD on the GPU; patches carrying their boundary cells, Sec. 3):
 *   hydro_mhd_step_patches: out[p] interior <- U^{n+1} of in[p] with time step dt_dev[p] (device
 *       array of npatch doubles) and cell size in[p].dx; in[p] and out[p] of equal sizes and dx, not
 *       overlapping; dt_next_dev: NULL or npatch doubles receiving each patch's CFL dt of U^{n+1}.
 *       HYDRO_FP32 and HYDRO_MIXED run one fused launch over tiles of 32 x 8 columns and 32 planes
 *       of every patch, with no per-cell scratch; HYDRO_FP64 and HYDRO_FP64_DF use device scratch of
 *       81 elements per cell of each patch's interior grown by one cell per side.
 *   hydro_mhd_cfl_patches: dt_dev[p] <- the CFL dt of each patch's interior (bit-identical to the
 *       fused one).
 * Precisions and errors as hydro_mhd_step.  The descriptors are uploaded when the patch set differs
 * from the previous call's (the stream is synchronised first). */
int hydro_mhd_step_patches(hydro_ctx* ctx, const hydro_mhd_patch* in, const hydro_mhd_patch* out, int npatch,
                           const double* dt_dev, double* dt_next_dev);
int hydro_mhd_cfl_patches(hydro_ctx* ctx, const hydro_mhd_patch* p, int npatch, double* dt_dev);

/* Adjoint of one step with dt held fixed (the paper has no adjoint; this is the reverse mode of
 * hydro_step):  lam_n = (dU^{n+1}/dU^n)^T lam_np1, for periodic boxes (ng == 0) in HYDRO_FP64,
 * HYDRO_FP64_DF (which runs the FP64 reverse sweep: faster on GB300 than a double-float one) or
 * HYDRO_FP32.  U_n: the
 * state the forward step started from; dt_dev[p] its time step; lam_np1, lam_n: adjoint fields
 * with the same layout and element type as U_n (must not overlap).  HYDRO_MIXED returns
 * HYDRO_ERR_ARG.  The
 * derivative of each limiter / HLLC branch / floor is that of the branch the forward values
 * select.  Deterministic: every face's contribution is gathered, never atomically scattered. */
int hydro_adjoint_step(hydro_ctx* ctx, const hydro_patch* U_n, const double* dt_dev, const hydro_patch* lam_np1,
                       const hydro_patch* lam_n, int npatch);

/* Primitive -> conservative map of the initial state and its adjoint (part of the adjoint interface,
 * no counterpart in the paper; the ideal-gas closure of Sec. 2; used to turn gradients with
 * respect to U^0 into gradients with respect to the initial density and velocity):
 *   U = (rho, rho u, rho v, rho w, p/(gamma-1) + rho |u|^2 / 2).
 * W holds (rho, u, v, w, p) in the layout of a patch; lamW receives (dU/dW)^T lamU. */
int hydro_prim_to_cons(hydro_ctx* ctx, const hydro_patch* W, const hydro_patch* U, int npatch);
int hydro_prim_to_cons_adjoint(hydro_ctx* ctx, const hydro_patch* W, const hydro_patch* lamU,
                               const hydro_patch* lamW, int npatch);

/* Multi-step run of one periodic box, each step at the adaptive time step of Sec. 2 and Sec. 4 (the
 * graph capture has no counterpart in the paper), with the time step kept on the device (no host
 * synchronisation per step): dt_hist_dev[0] = CFL dt of the state in a; step n advances by
 * dt_hist_dev[n] and writes dt_hist_dev[n+1] = CFL dt of its result; states ping-pong between
 * a (even n) and b (odd n), so the result is in a if nsteps is even, else in b.
 * dt_hist_dev: device array of nsteps + 1 doubles.  With use_graph != 0 the nsteps launches are
 * captured once into a CUDA graph (cached in the context for the same a, b, nsteps, dt_hist_dev)
 * and replayed. */
int hydro_run(hydro_ctx* ctx, const hydro_patch* a, const hydro_patch* b, int nsteps, double* dt_hist_dev,
              int use_graph);

/* One step of a periodic box whose state lives in HOST memory (the paper's GPU ports copy each
 * patch chunk to the GPU and back every step, and those copies cost a quarter of the GPU hydro time
 * and more, Sec. 3 and Table 1).  in->U / out->U are host pointers (page-locked memory lets the
 * copies run asynchronously; pageable memory works but serialises them), ng == 0, the same sy, sz
 * for in and out, and each field spans nz * sz elements.  The library stages the box in device
 * memory it owns (10 fields of nz * sz elements, kept for later calls) and pipelines the step over
 * z slabs: host->device copies on one stream, the step kernel on the context stream over each slab
 * whose halo planes have arrived, device->host copies of finished slabs on a third stream, so the
 * two transfers and the compute overlap.  dt_dev / dt_next_dev are DEVICE pointers as in
 * hydro_step (dt_next_dev, if not NULL, receives the CFL dt of the result).  The call returns once
 * the work is enqueued; out is complete when the context stream has been synchronised.  Device
 * pointers in in/out give HYDRO_ERR_ARG. */
int hydro_step_host(hydro_ctx* ctx, const hydro_patch* in, const hydro_patch* out, const double* dt_dev,
                    double* dt_next_dev);

/* Autotuner (no counterpart in the paper, whose Sec. 3 finds that small chunks starve the GPU): times
 * the candidate tile shapes and z-chunk depths of hydro_step on this patch set
 * (in, out, dt_dev as for hydro_step; contents of out are overwritten) and keeps the fastest in
 * the context for later hydro_step calls.  When a batch of ghosted patches holds patches of more
 * than one patch-shape class (below), it also times the candidates on each class's patches alone
 * and keeps a tile shape per class if the whole set then steps at least 1% faster (hydro_step then
 * runs one persistent launch per class).  If cache_path is not NULL the choice is read from /
 * appended to that text file, one line per tuning: the key (GPU name, SM count, precision,
 * limiter, patch-set signature), tile_id, zchunk, and tile_id, zchunk of each class (-1 0: the
 * context's).  Synchronises the stream. */
int hydro_autotune(hydro_ctx* ctx, const hydro_patch* in, const hydro_patch* out, int npatch, const double* dt_dev,
                   const char* cache_path);

/* Current tile configuration: *tile_id (index into the compiled tile shapes) and *zchunk (no
 * counterpart in the paper).  Compiled shapes (columns x rows of one block's tile): 0 16 x 16,
 * 1 32 x 8, 2 8 x 8, 3 32 x 16, 4 16 x 16 with a whole SM's registers for one block; the PPM
 * kernel has one shape (16 x 16) and ignores tile_id.  hydro_set_tuning refuses tile_id outside
 * [0, HYDRO_NUM_TILES) and zchunk outside [1, 4096]. */
#define HYDRO_NUM_TILES 5

/* Tile shape per patch-shape class of a batched hydro_step (no counterpart in the paper): the
 * classes are 0, a patch with an x or y edge of 8 cells or fewer; 1, else an x or y edge that is not
 * a multiple of 16; 2, both multiples of 16.  hydro_set_class_tuning(ctx, class, tile_id, zchunk)
 * gives a class its own tile shape and z chunk (tile_id -1: the context's, hydro_set_tuning's);
 * hydro_get_class_tuning returns the tuning a class's patches step with.  hydro_set_tuning resets
 * every class to the context's tuning.  A periodic box (ng == 0), the PPM kernel and the host-buffer
 * step use the context's tuning only.  HYDRO_ERR_ARG for a class outside [0,
 * HYDRO_NUM_PATCH_CLASSES) or a tuning hydro_set_tuning refuses. */
#define HYDRO_NUM_PATCH_CLASSES 3
int hydro_get_class_tuning(hydro_ctx* ctx, int patch_class, int* tile_id, int* zchunk);
int hydro_set_class_tuning(hydro_ctx* ctx, int patch_class, int tile_id, int zchunk);
int hydro_get_tuning(hydro_ctx* ctx, int* tile_id, int* zchunk);
int hydro_set_tuning(hydro_ctx* ctx, int tile_id, int zchunk);

/* Failure reporting (no counterpart in the paper): synchronise the context's stream and return the
 * device error word in *error_bits (may be
 * NULL).  Returns HYDRO_ERR_UNPHYSICAL if any bit is set, HYDRO_OK otherwise, HYDRO_ERR_CUDA on
 * a CUDA error.  hydro_clear_error zeroes the word (asynchronously). */
int hydro_get_error(hydro_ctx* ctx, unsigned* error_bits);
int hydro_clear_error(hydro_ctx* ctx);

/* Number of kernels this context has launched so far (graph replays count their kernels; no
 * counterpart in the paper). */
int hydro_launch_count(hydro_ctx* ctx, long long* count);

/* The batched step of hydro_step for callers that cannot allocate device memory (no counterpart
 * in the paper).  Some callers cannot call cudaMalloc: code running inside another runtime's
 * memory pool or a fixed memory budget, code that must not allocate after start-up, or a host
 * program that only receives device pointers.  hydro_step needs a context and hydro_init
 * allocates; this call needs none.  Its scratch -- uploaded patch descriptors, prefix-sum counts,
 * the tile work-list and the tile counter -- is a set of file-scope device arrays of fixed size
 * (about 4.7 MB) that every GPU loading the library holds until the process exits.  Limits:
 * npatch <= 4096 and at most 262144 tiles of 16 x 16 columns x 32 planes (HYDRO_ERR_ARG beyond
 * either).  cfg, in, out, npatch, dt_dev, dt_next_dev have the meaning of hydro_init's config and
 * hydro_step's arguments, with hydro_step's ghost rule (every input patch carries two ghost
 * layers; a single periodic box, ng == 0, none); the step runs the compiled tile 0 with 32-plane
 * z chunks, so its results are those of hydro_step at that tuning, bit for bit.  error_bits_dev
 * (required: NULL gives HYDRO_ERR_ARG) is a device word that receives HYDRO_EBIT_* bits by atomic
 * OR; the caller zeroes it and reads it back.  The first call on a device looks up the arrays' device
 * addresses (cudaGetSymbolAddress, with that device current): make that first call before any
 * stream capture.  Every call reuses the same arrays (their previous contents are overwritten;
 * the tile counter is cleared on each call), so calls whose work overlaps on the GPU -- on
 * different streams, or from different host threads -- race: serialise them.  Allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library call. */
int hydro_step_batched_noalloc(const hydro_config* cfg, const hydro_patch* in, const hydro_patch* out, int npatch,
                               const double* dt_dev, double* dt_next_dev, unsigned* error_bits_dev);

/* Static description of a status code (no counterpart in the paper). */
const char* hydro_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
