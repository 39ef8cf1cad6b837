/*
 * lbm.h -- C ABI of the GB300 sparse-geometry lattice Boltzmann library.
 *
 * One time step of the BGK lattice Boltzmann method (D2Q9, D3Q19) over a
 * uniform mesh of fixed-size tiles of which only the non-empty ones are
 * stored; every tile's fused stream+collide gathers its halo PDFs from its
 * neighbour tiles through a tile-index map.  This is the "tiles with two
 * copies" (T2C) method of Tomczak & Szafran, arXiv:1703.08015 (Sec. 3 and
 * Fig. 5), written for sm_103a.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: LBM_OK (0) or a negative
 *     LBM_ERR_* code.  No function aborts the process or traps the GPU.
 *     lbm_last_error() returns a message for the calling host thread.
 *   - Host masks and dense fields are laid out [z][y][x] with x fastest;
 *     2D lattices use nz = 1.  mask[n] != 0 marks a fluid node.
 *   - Dense PDF arrays are [i][z][y][x] (direction i slowest) in FP64 and
 *     hold post-collision values; the link order is the one documented at
 *     LBM_D2Q9 / LBM_D3Q19 below.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     stream-ordered; a context must not be used from two host threads at
 *     once.
 *   - The two device PDF buffers are allocated and freed by the caller (for
 *     example as PyTorch tensors) and only borrowed by the library; the small
 *     tables (tile masks, neighbour records, coordinates, reduction partials)
 *     are allocated by lbm_init and released by lbm_free.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBM_OK            0
#define LBM_ERR_ARG      (-1) /* bad argument: NULL pointer, size, lattice, tau <= 1/2 */
#define LBM_ERR_SHAPE    (-2) /* a periodic axis is not a multiple of tile_a */
#define LBM_ERR_CUDA     (-3) /* a CUDA runtime call failed */
#define LBM_ERR_OOM      (-4) /* a device allocation failed */
#define LBM_ERR_DIVERGED (-5) /* the mass or momentum sum is not finite */
#define LBM_ERR_TIMEOUT  (-6) /* a bounded device-side wait ran out */
#define LBM_ERR_BOUNDS   (-7) /* a checked kernel saw an index outside its buffers */
#define LBM_ERR_CAPACITY (-8) /* a request exceeds a fixed capacity */

/* ---- lattices ----------------------------------------------------------
 * LBM_D2Q9  links: 0 (0,0); 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1);
 *                  5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1).
 *           weights 4/9, 1/9 (links 1-4), 1/36 (links 5-8).
 * LBM_D3Q19 links: 0 (0,0,0); 1 +x 2 -x 3 +y 4 -y 5 +z 6 -z;
 *                  7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *                  11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1)
 *                  15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1).
 *           weights 1/3, 1/18 (links 1-6), 1/36 (links 7-18).
 * The paper names both lattices (Fig. 1, Sec. 2.2) without printing either
 * table; these are the standard sets. */
#define LBM_D2Q9   9
#define LBM_D3Q19 19

/* Equilibrium model: Eq. 3 with Eq. 5 (quasi-compressible) or Eq. 4 with
 * Eq. 6 (incompressible). */
#define LBM_QUASI_COMPRESSIBLE 0
#define LBM_INCOMPRESSIBLE     1

/* PDF storage in device memory.  LBM_STORE_F64 is the FP64 method of the
 * paper (all of its runs are double precision, Sec. 4). */
#define LBM_STORE_F64  0
#define LBM_STORE_F32  1 /* FP32 values, FP32 collision (not in the paper) */
#define LBM_STORE_F16S 2 /* FP16 scaled deviations (f_i - w_i) * S, FP32 collision (not in the paper) */
#define LBM_STORE_F32S 3 /* FP32 deviations f_i - w_i, FP32 collision (not in the paper) */

/* Arithmetic of the FP64 step.  All variants compute the same FP64 update;
 * they differ only in rounding (see lbm_step).  Nodes outside the range of
 * the fixed-point and float-float forms fall back to native FP64. */
#define LBM_ARITH_AUTO   0 /* LBM_ARITH_FF (the default) */
#define LBM_ARITH_F64    1 /* native FP64 instructions */
#define LBM_ARITH_FIXED  2 /* exact 64-bit fixed-point sums and products, no FP64 instructions */
#define LBM_ARITH_FF     3 /* exact integer sums, float-float products (~48 bits), no FP64 instructions;
                              the tile-map gather of Fig. 5 (neighbourhood staged per block) */
#define LBM_ARITH_FF_TABLE 4 /* LBM_ARITH_FF with each node's sources read from a per-node
                              gather table built once: the connectivity-matrix scheme of
                              Sec. 2.3.1 (Eqs. 13-14) on the compact tiles, not the tile-map
                              method; 4 (q + 1) bytes per fluid node more per step */

/* PDF layouts (Sec. 3.1).  T2C: two copies, each step reads one and writes the
 * other (Fig. 5).  TGB: one copy updated in place; values that cross a tile
 * edge travel through two sets of ghost buffers (per tile and link, the nodes
 * on the tile's downstream boundary), so the memory is one copy plus the
 * ghost sets (lbm_tiling.ghost_bytes).  The update is the same bit for bit. */
#define LBM_LAYOUT_T2C 0
#define LBM_LAYOUT_TGB 1

/* lbm_moments flags */
#define LBM_OUT_DEVICE    1 /* rho/u/pdf pointers are device pointers (default: host) */
#define LBM_STATS_RESIDUAL 2 /* compute the steady-state residual against the
                                velocity saved by the previous residual call,
                                then save the current velocity */

typedef struct lbm_params {
    int lattice;      /* LBM_D2Q9 or LBM_D3Q19 */
    int model;        /* LBM_QUASI_COMPRESSIBLE or LBM_INCOMPRESSIBLE */
    int nx, ny, nz;   /* lattice size; nz = 1 for D2Q9 */
    int tile_a;       /* nodes per tile edge a (Sec. 3): D2Q9 8, 16, 32; D3Q19 4, 8 */
    int periodic[3];  /* per axis: 1 = periodic (length must be a multiple of a),
                         0 = solid wall halfway outside the last node row */
    double tau;       /* BGK relaxation time (Eq. 2), > 1/2; viscosity (tau - 1/2)/3 */
    double force[3];  /* body-force density F (Guo forcing; not in the paper) */
    double rho0;      /* density of the rest start (used when no rho field is given) */
    int storage;      /* LBM_STORE_* */
    int arith;        /* LBM_ARITH_* (LBM_STORE_F64 only) */
    double f16_scale; /* LBM_STORE_F16S: scale S of the deviations (a power of two
                         keeps the scaling exact); 0 = default 2^16 */
    int block_nodes;  /* fluid nodes per step-kernel block: 0 = default (256, or a^d
                         when a tile has more nodes; 128 for the LBM_ARITH_FF /
                         LBM_ARITH_AUTO FP64 step with 4^3 / 8^2 tiles); 128 is
                         also compiled for the FP32 storage forms with 4^3 / 8^2
                         tiles (autotuner choice); other values: LBM_ERR_ARG */
    int persistent;   /* 1 = FP32 storage forms run a persistent step kernel: as many
                         blocks as fit on the GPU at once loop over the work list */
    int layout;       /* LBM_LAYOUT_T2C (two PDF copies, default) or LBM_LAYOUT_TGB
                         (one copy updated in place plus ghost buffers, Sec. 3.1) */
    int prefetch_blocks; /* not in the paper: in the float-float FP64 step on tiles of
                         one mask word (4^3, 8^2) and the FP32 storage forms' step
                         (LBM_LAYOUT_T2C, not persistent), each block asks the L2 for
                         the source values of the work block this many blocks ahead,
                         so that its gathers find them there (the FP32 forms also for
                         that block's node list and neighbour indices); 0 = default
                         (4 per SM), < 0 = off.  Timing only: results do not depend
                         on it */
} lbm_params;

typedef struct lbm_tiling {
    int32_t ntx, nty, ntz; /* tile mesh (ntz = 1 in 2D) */
    int32_t n_tiles;       /* N_tiles = ntx * nty * ntz (Sec. 3.1.1.1) */
    int32_t n_ftiles;      /* N_ftiles, the non-empty tiles */
    int32_t nbr_per_tile;  /* 3^d entries in each neighbour record */
    int64_t n_fluid;       /* N_fnodes, non-solid nodes (Eq. 11) */
    size_t pdf_bytes;      /* bytes of ONE PDF copy in the requested storage */
    size_t ghost_bytes;    /* LBM_LAYOUT_TGB: bytes of the two ghost-buffer sets that
                              pdf_b must hold (0 for LBM_LAYOUT_T2C) */
} lbm_tiling;

typedef struct lbm_stats {
    double mass;        /* sum over fluid nodes of rho */
    double momentum[3]; /* sum over fluid nodes of rho u (u with the F/2 correction) */
    double u2;          /* sum over fluid nodes of |u|^2 */
    double du2;         /* sum of |u - u_saved|^2 (LBM_STATS_RESIDUAL) */
    double residual;    /* sqrt(du2 / u2); +inf when no velocity was saved yet */
    int64_t n_fluid;    /* fluid nodes summed */
    int64_t step;       /* time steps taken since lbm_init */
} lbm_stats;

typedef struct lbm_ctx lbm_ctx; /* opaque; owned by the library */

/* Tile the geometry (Sec. 3): cover it with a x a (x a) tiles starting at
 * node (0,0), pad with solid nodes, drop the tiles that hold only solid
 * nodes, and number the others by their rank in row-major scan order
 * (x fastest).  Host only, no device work.
 *   p         lattice, nx, ny, nz, tile_a, periodic and storage are read.
 *   mask      host, nx*ny*nz bytes, [z][y][x], nonzero = fluid.
 *   tile_map  host out, n_tiles int32 [tz][ty][tx]: the tile's index or -1
 *             for a removed tile (the tileMap of Sec. 3); NULL = size query.
 *   nbr       host out, n_ftiles * 3^d int32: for each non-empty tile the
 *             index of each surrounding tile, offsets (dz, dy, dx) in
 *             {-1,0,1} with dx fastest, -1 for a removed tile or one beyond
 *             a non-periodic edge (the 3^3 tile bitmap of Fig. 5); NULL =
 *             not wanted.  Its size is only known after a size query.
 *   out       host out, the counts and the bytes of one PDF copy.
 * The mask scan and the neighbour records run over tile rows in up to 16
 * host threads (the result does not depend on their number); lbm_init tiles
 * the same way and builds the same neighbour records on the device.
 * Errors: LBM_ERR_ARG (NULL mask/out/p, bad sizes or tile edge),
 * LBM_ERR_SHAPE (periodic axis not a multiple of tile_a), LBM_ERR_CAPACITY
 * (too many tiles; with nbr given, neighbours more than 2^30 values apart,
 * which lbm_init reports in any case). */
int lbm_build_tilemap(const lbm_params* p, const uint8_t* mask,
                      int32_t* tile_map, int32_t* nbr, lbm_tiling* out);

/* Create a context: tile the mask, upload the tile tables, and fill PDF copy
 * A with the equilibrium f^eq(rho, u) of Eq. 3 (Eq. 4 for the incompressible
 * model) at every fluid node, zero elsewhere.
 *   out        receives the context (NULL on failure).
 *   mask       host, as in lbm_build_tilemap.
 *   pdf_a/b    device, caller-owned, each at least `pdf_bytes` bytes and
 *              256-byte aligned; they must stay allocated until lbm_free.
 *              With LBM_LAYOUT_TGB, pdf_a is the copy (`pdf_bytes`) and pdf_b
 *              holds the ghost sets (at least lbm_tiling.ghost_bytes).
 *   rho_init   dense nx*ny*nz doubles, or NULL for rho0 everywhere; device
 *              memory of the current device is read in place (it must stay
 *              valid until the fill on `stream` has run), other memory
 *              (host, another device) is copied first.
 *   u_init     dense 3 * nx*ny*nz doubles [component][z][y][x] (2 * ... for
 *              D2Q9), or NULL for rest; memory as for rho_init.
 *   stream     cudaStream_t on which the uploads and the fill run; the call
 *              returns after they have been issued (tables copied from host
 *              memory synchronously).
 * Errors: LBM_ERR_ARG, LBM_ERR_SHAPE, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_init(lbm_ctx** out, const lbm_params* p, const uint8_t* mask,
             void* pdf_a, void* pdf_b, size_t pdf_bytes,
             const double* rho_init, const double* u_init, void* stream);

/* Advance `nsteps` time steps of Eq. 7 with the Eq. 2 BGK collision: each
 * non-empty tile gathers the post-collision values f*_i(r - c_i) of its own
 * and its neighbour tiles through the neighbour record (Fig. 5), takes its
 * own f*_{opp(i)}(r) where r - c_i is solid, empty or beyond a wall
 * (propagation only between non-solid nodes, Sec. 3.2: halfway bounce-back),
 * collides, and stores into the other copy; the copies then swap (Sec. 3).
 * Asynchronous on `stream`.  With LBM_ARITH_FIXED the FP64 update is computed
 * with 64-bit fixed-point integers (resolution 2^-60), with LBM_ARITH_FF
 * with exact integer sums and float-float products; either is rounded once to
 * FP64 and agrees with LBM_ARITH_F64 to rounding.  LBM_ARITH_AUTO is
 * LBM_ARITH_FF.  LBM_ARITH_FF_TABLE is the float-float update with the gather
 * resolved once, the connectivity-matrix scheme the paper compares against
 * (Sec. 2.3.1): lbm_init builds a table of every node's source slots
 * (4 (q + 1) bytes per fluid node, allocated by the library, T2C layout,
 * when the copy's value indices fit int32; else the staged gather of
 * LBM_ARITH_FF), and the step reads it instead of staging the neighbourhood.
 * Errors: LBM_ERR_ARG (NULL ctx, nsteps < 0), LBM_ERR_CUDA. */
int lbm_step(lbm_ctx* ctx, int nsteps, void* stream);

/* Density and velocity that the next step will collide with (the gathered
 * values; rho = sum f_i, u from Eq. 5 / Eq. 6 with the F/2 correction), and
 * FP64 reductions over the fluid nodes in a fixed order (deterministic; for a
 * batch the sums run over all samples, in sample order).
 *   rho    dense nx*ny*nz doubles or NULL (single geometry only); NaN at solid.
 *   u      dense 3*nx*ny*nz doubles [component][z][y][x] or NULL; NaN at solid.
 *   stats  host, or NULL.
 *   flags  LBM_OUT_DEVICE: rho and u are device pointers (default host);
 *          LBM_STATS_RESIDUAL: fill stats->du2 and stats->residual.
 * Synchronises `stream` when anything is returned to host memory.
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_DIVERGED (mass or momentum not
 * finite; stats is still filled). */
int lbm_moments(lbm_ctx* ctx, double* rho, double* u, lbm_stats* stats,
                int flags, void* stream);

/* Copy the current post-collision PDFs out as a dense FP64 array
 * [i][z][y][x] (q * nx*ny*nz doubles; solid nodes NaN), host or device
 * (LBM_OUT_DEVICE).  Used for checkpoints and for checking the step.  Single
 * geometry only (a batch uses lbm_export_pdfs_sample).
 * Synchronises `stream` for host output.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_export_pdfs(lbm_ctx* ctx, double* pdfs, int flags, void* stream);

/* Overwrite the current post-collision PDFs from a dense FP64 array laid out
 * as in lbm_export_pdfs (values at solid nodes are ignored; single geometry
 * only); `step` becomes
 * the context's step count.  Resuming from an exported state reproduces an
 * uninterrupted run bit for bit.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_import_pdfs(lbm_ctx* ctx, const double* pdfs, int64_t step, int flags,
                    void* stream);

/* Largest number of partial-sum blocks lbm_stats_noalloc can hold: its
 * static scratch is LBM_NOALLOC_MAX_BLOCKS * 8 doubles (512 KiB) per GPU. */
#define LBM_NOALLOC_MAX_BLOCKS 8192

/* The mass and momentum sums of lbm_moments without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they want the sums -- code working inside a
 * fixed device-memory budget owned by another allocator, monitoring hooks
 * that must not change the memory footprint between steps, or loops that
 * cannot afford the device-wide synchronisation cudaMalloc implies.
 *   ctx        a context from lbm_init (its tables were allocated there).
 *   stats_dev  device, caller-allocated, 8 doubles: on completion
 *              [mass, momentum x, y, z, sum |u|^2, 0, fluid-node count, 0]
 *              with the meanings of lbm_stats; no residual.
 *   stream     cudaStream_t; the call only enqueues work (nothing is copied
 *              to the host and the stream is not synchronised).
 * The per-block partial sums go to a file-scope device array of
 * LBM_NOALLOC_MAX_BLOCKS * 8 doubles that every GPU loading the library
 * keeps until the process exits.  One partial block covers 32 non-empty
 * tiles of 4^3 or 8^2 nodes, or 8 tiles of 8^3, 16^2 or 32^2 nodes, so
 * tilings that need more than LBM_NOALLOC_MAX_BLOCKS blocks (more than
 * 262,144 non-empty 4^3 tiles, for example) are rejected with
 * LBM_ERR_CAPACITY.  The device that was current at lbm_init must be current
 * (else LBM_ERR_ARG).  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any
 * stream capture.  A cudaDeviceReset invalidates that address: calls after
 * one are not supported.  All calls share the one array, which keeps the
 * last call's contents: every block writes its slots before they are read,
 * so nothing has to start at zero, but calls whose kernels overlap on the
 * GPU race with each other.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: LBM_ERR_ARG, LBM_ERR_CAPACITY, LBM_ERR_CUDA. */
int lbm_stats_noalloc(const lbm_ctx* ctx, double* stats_dev, void* stream);

/* ---- batches of geometries (not in the paper) ------------------------------
 * Many independent samples of uneven size and sparsity advance together: each
 * sample is tiled on its own and the tiles of all samples form one
 * concatenated list (one work list, one launch per step; with
 * params->persistent a grid of resident blocks loops over it).  lbm_step
 * applies to a batch unchanged; moments and exports are per sample.  All
 * samples share params (lattice, tile edge, periodic axes, tau, force,
 * storage); params->nx/ny/nz are ignored.
 *   dims   host, n_samples * 3 ints: nx, ny, nz of each sample.
 *   masks  host, n_samples pointers to [z][y][x] masks (nonzero = fluid). */

/* Counts summed over the samples and the bytes of one PDF copy of the batch.
 * Errors: LBM_ERR_ARG, LBM_ERR_SHAPE (a sample's periodic axis), LBM_ERR_CAPACITY. */
int lbm_build_tilemap_batch(const lbm_params* p, int n_samples, const int* dims,
                            const uint8_t* const* masks, lbm_tiling* out);

/* Like lbm_init for a batch (every sample starts at rest with density rho0).
 * Errors: as lbm_init. */
int lbm_init_batch(lbm_ctx** out, const lbm_params* p, int n_samples, const int* dims,
                   const uint8_t* const* masks, void* pdf_a, void* pdf_b, size_t pdf_bytes,
                   void* stream);

/* Per-sample statistics: stats[k] for sample k (as lbm_moments; the residual
 * uses each sample's own sums).  Synchronises `stream`.
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_DIVERGED (some sample). */
int lbm_moments_batch(lbm_ctx* ctx, lbm_stats* stats, int flags, void* stream);

/* The rho / u fields of lbm_moments for sample k of a batch (dense over that
 * sample's box, NaN at solid nodes; host or device with LBM_OUT_DEVICE).
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_moments_sample(lbm_ctx* ctx, int sample, double* rho, double* u, int flags, void* stream);

/* Period-2 filter for steady-state runs (not in the paper).  Replaces the
 * current post-collision state by the mean of it and the state one step
 * earlier (the other PDF copy), word by word in the storage format:
 * f <- (f(t) + f(t-1)) / 2.
 *
 * The BGK step with halfway bounce-back has a slowly damped mode that flips
 * sign every step (a staggered, checkerboard pattern of the velocity along the
 * links).  Starts from rest or from a predicted field excite it; a residual
 * taken over an even number of steps does not see it flip, only its slow decay
 * (the factor per step is close to -1), so it both delays the test of a
 * steady state and is still present, at a relative velocity error near 1e-3,
 * when that test passes.  The mean of two consecutive states removes it and
 * leaves every slowly varying part of the state, so the fixed point of the
 * update is unchanged.  Needs at least one lbm_step since lbm_init,
 * lbm_import_pdfs or the last filter (the other copy must hold the previous
 * state); applies to every sample of a batch.  Asynchronous on `stream`.
 * Errors: LBM_ERR_ARG (NULL ctx, no previous state), LBM_ERR_CUDA. */
int lbm_filter_period2(lbm_ctx* ctx, void* stream);

/* lbm_export_pdfs for sample k of a batch (dense over that sample's box).
 * Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
int lbm_export_pdfs_sample(lbm_ctx* ctx, int sample, double* pdfs, int flags, void* stream);

/* ---- tile layers: the domain split across GPUs (not in the paper) ----------
 * The paper names multi-GPU runs as future work (Sec. 5).  A geometry split
 * into slabs of whole tile layers along its slowest tile axis (z in 3D, y in
 * 2D) runs one context per GPU on the rank's box: its slab plus one ghost
 * tile layer on each side that has a neighbour.  Tiles are numbered
 * row-major with that axis slowest, so the non-empty tiles of a run of
 * layers are consecutive and their values form one contiguous range of a
 * PDF copy; the same layer of the same mask has the same bytes in any
 * context.  After every step a rank copies its first and last interior
 * layers into the neighbours' ghost layers (NCCL send/recv into the
 * receiver's memory) and the split run matches the undivided one bit for
 * bit.  Single-geometry T2C contexts only (LBM_ERR_ARG otherwise). */

/* Byte offset and length, within either PDF copy, of the non-empty tiles of
 * the tile layers [l_begin, l_end).  Host only, no device work.
 * Errors: LBM_ERR_ARG (NULL arguments, layers out of range, batch or TGB). */
int lbm_layer_range(const lbm_ctx* ctx, int l_begin, int l_end, size_t* offset, size_t* bytes);

/* Which of the two PDF buffers given to lbm_init (0 = pdf_a, 1 = pdf_b)
 * holds the current post-collision state, as of the work enqueued so far;
 * -1 for NULL. */
int lbm_current_copy(const lbm_ctx* ctx);

/* lbm_moments' statistics restricted to the fluid nodes of the tile layers
 * [l_begin, l_end) (a rank's interior), reduced in a fixed order; flags
 * LBM_STATS_RESIDUAL as in lbm_moments (the saved velocity covers those
 * layers).  Synchronises `stream`.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA,
 * LBM_ERR_DIVERGED. */
int lbm_moments_layers(lbm_ctx* ctx, int l_begin, int l_end, lbm_stats* stats, int flags, void* stream);

/* Number of samples in the context (1 for lbm_init); 0 for NULL. */
int lbm_num_samples(const lbm_ctx* ctx);

/* Counts of the context's tiling (see lbm_tiling).  Errors: LBM_ERR_ARG. */
int lbm_get_tiling(const lbm_ctx* ctx, lbm_tiling* out);

/* Release the context and the tables lbm_init allocated for it -- the tile
 * map, neighbour records and node types of Sec. 3 / Fig. 5, the work list,
 * the reduction partials -- but never the caller's PDF buffers.  Waits for
 * the context's pending work (cudaDeviceSynchronize).  NULL is accepted.
 * Errors: LBM_ERR_CUDA (a pending kernel failed; the context is still
 * released). */
int lbm_free(lbm_ctx* ctx);

/* Message describing the last failure on the calling host thread. */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
