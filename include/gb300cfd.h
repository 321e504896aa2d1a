/* gb300cfd — explicit staggered-grid incompressible Navier-Stokes time step
 * on GB300 (sm_103a), behind a plain C ABI.
 *
 * The method is the 3D CFD demonstration code of Blazewicz et al.,
 * "A Massive Data Parallel Computational Framework for Petascale/Exascale
 * Hybrid Computer Systems": Navier-Stokes with modified pressure phi = p/rho
 * (Sec. 4.1, Eq. 1) and incompressibility (Eq. 2), finite differences on a
 * regular rectangular staggered grid (Sec. 4.1), explicit Runge-Kutta Method
 * of Lines time integration (Sec. 1), block-structured grid components with
 * ghost regions of run-time width filled by copy from the neighbouring
 * component or from the physical boundary condition (Sec. 1.1), and a
 * velocity update u <- u - (dt/rho) grad p with separate in/out velocity
 * buffers (the UPDATE_VELOCITY kernel descriptor of Sec. 3, Listing 1).
 *
 * Discretisation (where the paper is silent):
 *   MAC placement, cell (i,j,k) of size h = (hx,hy,hz):
 *     p at ((i+1/2)hx,(j+1/2)hy,(k+1/2)hz); u, v, w on the +x, +y, +z faces.
 *   F(u) = -(u . grad) u + nu lap u, advective form, central differences;
 *     order 2 (ghost >= 1) or order 4 (ghost = 2); or (cfd_set_advection)
 *     the conservative form -div(u u) + nu lap u, order 2.
 *   Heun RK2, each stage projected:
 *     stage 1: w = u^n + dt F(u^n),              c = 1
 *     stage 2: w = 1/2 u^n + 1/2 u1 + 1/2 dt F(u1), c = 1/2
 *     r = (D w)/(c dt);  p <- K weighted Jacobi sweeps of L p = r (warm start),
 *     or V-cycles of a geometric multigrid (cfd_set_pressure_solver);
 *     u_next = w - c dt G p.
 *
 * Conventions for every entry point:
 *   - Return value is a cfd_status; no call aborts, exits or throws.  On an
 *     error, cfd_last_error() returns a message (a per-thread copy).
 *   - Work is enqueued asynchronously on the grid's stream (the stream given
 *     at creation; 0 means the legacy default stream).  Internally the
 *     library runs on a private stream joined to the caller's stream with
 *     events on entry and exit, so ordering with the caller's own work on
 *     that stream is preserved.  Calls that return host values
 *     (cfd_reduce, cfd_residual, cfd_check) synchronise.
 *   - CFD_ECUDA is sticky: after an asynchronous CUDA error the grid refuses
 *     further work.
 *   - Arrays: one array per field and block, storage type chosen at creation
 *     (FP32, BF16 or FP16; arithmetic is always FP32, global reductions FP64).
 *     Layout: (nz+2g) planes x (ny+2g) rows x row pitch, x fastest; the
 *     interior x = 0 of every row is 128-byte aligned.  cfd_array_layout()
 *     gives the exact offsets.  Device memory is either bound by the caller
 *     (cfd_bind_memory; the library never frees it) or allocated by the
 *     library (cfd_alloc_memory; freed by cfd_grid_destroy).
 */
#ifndef GB300CFD_H
#define GB300CFD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cfd_grid cfd_grid;

typedef enum {
  CFD_OK = 0,
  CFD_EINVAL = 1,        /* bad argument (sizes, pointers, face/array ids) */
  CFD_ENOMEM = 2,        /* bound memory too small / allocation failed */
  CFD_ECUDA = 3,         /* a CUDA call failed (sticky) */
  CFD_ESTATE = 4,        /* call out of order (no memory bound, ...) */
  CFD_EUNSUPPORTED = 5,  /* valid but not implemented combination */
  CFD_ENONFINITE = 6,    /* a reduction met NaN or Inf */
  CFD_ETIMEOUT = 7       /* a bounded device wait gave up (device error flag) */
} cfd_status;

typedef enum { CFD_F32 = 0, CFD_BF16 = 1, CFD_F16 = 2 } cfd_dtype;

/* Face kinds.  PERIODIC: ghost cells copy the opposite side (or, in a block
 * set, the neighbouring block).  WALL: no-slip wall moving with a given
 * tangential velocity: the wall-normal velocity is zero (the normal face
 * unknown on the high side is held at 0), tangential ghosts are
 * 2 U_wall - first interior, pressure ghosts copy the first interior
 * (zero normal gradient).  Sec. 1.1: physical boundaries are set from
 * boundary conditions, internal ones copied from neighbours. */
typedef enum { CFD_BC_PERIODIC = 0, CFD_BC_WALL = 1 } cfd_bc;

/* Form of the advection term of the momentum equation (Sec. 4.1, Eq. 1). */
typedef enum {
  CFD_ADVECTIVE = 0,  /* (u . grad) u_c, central differences (default) */
  CFD_FLUX = 1        /* div(u u_c), the conservative form (order 2) */
} cfd_advection;

/* Array ids.  State: U, V, W (velocity) and P (pressure, also the Jacobi
 * warm start).  Work arrays: WU..WW (provisional stage velocity), U1..W1
 * (stage-1 velocity), P2 (Jacobi ping-pong), R (Poisson right-hand side).
 * Adjoint state: LU, LV, LW, LP = dL/du, dL/dv, dL/dw, dL/dp. */
typedef enum {
  CFD_U = 0, CFD_V = 1, CFD_W = 2, CFD_P = 3,
  CFD_WU = 4, CFD_WV = 5, CFD_WW = 6,
  CFD_U1 = 7, CFD_V1 = 8, CFD_W1 = 9,
  CFD_P2 = 10, CFD_R = 11,
  CFD_LU = 12, CFD_LV = 13, CFD_LW = 14, CFD_LP = 15,
  CFD_NUM_ARRAYS = 16
} cfd_array;

/* Velocity triples for cfd_stage / cfd_project / cfd_reduce. */
typedef enum { CFD_SET_U = 0, CFD_SET_W = 1, CFD_SET_U1 = 2 } cfd_vset;

/* ---------------------------------------------------------------- set-up */

/* One block of dims[0] x dims[1] x dims[2] interior cells (x, y, z), ghost
 * width 1 or 2 (Sec. 1.1: chosen at run time), cell size h (> 0), storage
 * dtype.  All faces start PERIODIC.  dims[d] >= 2*ghost.  stream is a
 * cudaStream_t (may be NULL).  *out receives the handle. */
cfd_status cfd_grid_create(const int dims[3], int ghost, const double h[3], int storage,
                           void* stream, cfd_grid** out);

/* nblocks blocks tiling the periodic box global_dims exactly as a
 * rectilinear (slab-product) tiling: dims and origin are nblocks*3 ints
 * (x,y,z per block).  Ghost cells are copied from the neighbouring block
 * (Sec. 1.1: the driver's ghost exchange between grid components, here an
 * on-device copy).  Every block needs dims[d] >= 2*ghost. */
cfd_status cfd_blockset_create(int nblocks, const int* dims, const int* origin,
                               const int global_dims[3], int ghost, const double h[3],
                               int storage, void* stream, cfd_grid** out);

/* Releases the grid (and memory from cfd_alloc_memory).  Waits for the
 * grid's queued work.  A null grid is a no-op (CFD_OK); every other call
 * returns CFD_EINVAL for a null grid. */
cfd_status cfd_grid_destroy(cfd_grid* g);

/* Device bytes needed for all arrays of all blocks plus the library's
 * tables and reduction scratch (and, on single FP32 blocks whose dims
 * halve at least once, the multigrid levels: 1/7 of one field). */
cfd_status cfd_memory_bytes(const cfd_grid* g, size_t* bytes);

/* Binds caller-owned device memory (>= cfd_memory_bytes, 256-byte aligned).
 * The caller keeps ownership and must keep it alive until destroy. */
cfd_status cfd_bind_memory(cfd_grid* g, void* dev_ptr, size_t bytes);

/* Allocates the memory with cudaMalloc instead (owned by the grid). */
cfd_status cfd_alloc_memory(cfd_grid* g);

/* Layout of one array of one block: byte offset of element (-g,-g,-g)
 * from the bound base, shape (z, y, x) including ghosts, strides in
 * elements (z, y, x), and element size in bytes. */
cfd_status cfd_array_layout(const cfd_grid* g, int block, int array, long long* offset_bytes,
                            long long shape[3], long long strides[3], int* elem_bytes);

/* Number of blocks, ghost width and interior dims of a block. */
cfd_status cfd_block_info(const cfd_grid* g, int block, int dims[3], int origin[3], int* ghost);

/* Face 0..5 = -x,+x,-y,+y,-z,+z.  Periodic faces come in pairs; WALL needs
 * a single-block grid; the normal component of wall_velocity must be 0
 * (may be NULL for a still wall). */
cfd_status cfd_set_bc(cfd_grid* g, int face, int kind, const double wall_velocity[3]);

/* Physical and solver parameters: viscosity nu >= 0, Jacobi sweeps per
 * solve (>= 0), Jacobi weight omega in (0, 2), stencil order 2 or 4
 * (order 4 needs ghost 2). */
cfd_status cfd_set_params(cfd_grid* g, double nu, int jacobi_iters, double omega, int order);

/* Form of the advection term used by cfd_rhs_eval, cfd_stage and the steps.
 * CFD_ADVECTIVE (default): -(u . grad) u_c with the transverse velocity
 * interpolated to the point of u_c.  CFD_FLUX: -div(u u_c), which Eq. 2
 * (div u = 0) makes equal to the advective term for the continuous field:
 * around the point of u_c the flux through the side normal to axis d is
 * the product of the means of u_c and u_d nearest that side, and the term is
 * the flux difference over h_d.  Its sum over a periodic grid vanishes for
 * every field (momentum conservation) and, for a discretely divergence-free
 * field, so does the work sum u_c A_c (energy conservation).  CFD_FLUX is
 * order 2 only (CFD_EINVAL with order 4, here or in cfd_set_params later);
 * the adjoint (cfd_adjoint_step, cfd_rollout_*) linearises either form.
 * Invalidates captured step graphs. */
cfd_status cfd_set_advection(cfd_grid* g, int form);

/* ------------------------------------------------------ steps of the path */

/* Fill ghost cells of the arrays in mask (bit = 1 << cfd_array) on every
 * block: periodic/neighbour copy or wall rule, axis passes x then y then z
 * over the full extent (a later pass wins on edges and corners).  Sec. 1.1. */
cfd_status cfd_ghost_fill(cfd_grid* g, unsigned mask);

/* out = a * X + b * Y + c * F(Y) on the interior, F(u) = -(u.grad)u + nu lap u
 * (Eq. 1 without pressure, f = 0).  Y needs filled ghosts; wall-normal
 * faces of out are set to 0; out's ghosts are not filled.  x_set is ignored
 * when a == 0.  out must differ from x_set and y_set. */
cfd_status cfd_stage(cfd_grid* g, double a, int x_set, double b, int y_set, double c,
                     int out_set);

/* Residual-controlled variant of cfd_pressure_solve (an extension: the
 * paper's step uses a fixed sweep count): R = (D W)/c_dt, then weighted
 * Jacobi sweeps on P in chunks of check_every until ||L P - R||_2 <=
 * rtol ||R||_2 (checked before the first chunk and after each) or
 * max_iters sweeps.  iters_done and residual (either may be NULL) receive
 * the sweeps taken and the last ||L P - R||_2.  Synchronises once per
 * chunk; the residual is taken per cell in float-float and summed in FP64. */
cfd_status cfd_pressure_solve_converged(cfd_grid* g, double c_dt, double rtol, int max_iters,
                                        int check_every, int* iters_done, double* residual);

/* Geometric multigrid for the pressure equation L P = R (an extension: the
 * paper fixes no solver).  Cell-centred V-cycle in the correction scheme:
 * level l + 1 halves every axis of level l (coarse cell I covers fine cells
 * 2I and 2I + 1) and keeps the faces' kinds; every level uses the 7-point
 * L with its own cell size 2^l h; smoother: weighted Jacobi of weight omega
 * (nu1 sweeps before, nu2 after the coarse correction, ncoarse on the
 * coarsest level); restriction: mean over the 8 fine cells of R - L P;
 * prolongation: trilinear interpolation of the coarse correction at the
 * fine cell centres (weights 3/4, 1/4 per axis, coarse ghosts at faces).
 * Single FP32 blocks whose dims are even down to the coarsest level: the
 * grid keeps three arrays per level (1/7 of one field in total) in its
 * memory (cfd_memory_bytes includes them). */

/* Coarse levels available: halvings while every dim is even and >= 4
 * (0 for block sets, 16-bit storage or odd dims). */
cfd_status cfd_multigrid_levels(const cfd_grid* g, int* levels);

/* Cycle parameters: levels (0 = all available, else 1..available), nu1,
 * nu2 >= 0, ncoarse >= 1, omega in (0, 2).  Defaults 0, 2, 2, 30, 6/7.
 * CFD_EINVAL on a bad value. */
cfd_status cfd_set_multigrid(cfd_grid* g, int levels, int nu1, int nu2, int ncoarse,
                             double omega);

/* cycles V-cycles on P for L P = R as they stand (P's ghosts must be
 * filled; they are on exit).  Asynchronous on the grid's stream.
 * CFD_EUNSUPPORTED where cfd_multigrid_levels is 0. */
cfd_status cfd_mg_vcycles(cfd_grid* g, int cycles);

/* R = (D W)/c_dt, then V-cycles on P (warm start) until ||L P - R||_2 <=
 * rtol ||R||_2 (checked before the first cycle and after each) or
 * max_cycles.  cycles_done and residual (either may be NULL) receive the
 * cycles taken and the last ||L P - R||_2.  Synchronises once per cycle. */
cfd_status cfd_pressure_solve_mg(cfd_grid* g, double c_dt, double rtol, int max_cycles,
                                 int* cycles_done, double* residual);

/* Pressure solve inside the steps' stages (cfd_rk_step, cfd_step):
 * CFD_SOLVER_JACOBI (default) takes jacobi_iters sweeps (cfd_set_params);
 * CFD_SOLVER_MG takes 'cycles' (>= 1) V-cycles of cfd_set_multigrid's
 * parameters, warm-started from the last pressure.  CFD_EUNSUPPORTED for
 * CFD_SOLVER_MG where cfd_multigrid_levels is 0; the adjoint needs
 * CFD_SOLVER_JACOBI.  Invalidates captured step graphs. */
typedef enum { CFD_SOLVER_JACOBI = 0, CFD_SOLVER_MG = 1 } cfd_solver;
cfd_status cfd_set_pressure_solver(cfd_grid* g, int solver, int cycles);

/* F(U) = -(U . grad) U + nu lap U (Eq. 1 without the pressure term, f = 0;
 * the form of cfd_set_advection), U's ghosts filled, wall-normal faces 0:
 * always into WU, WV, WW (cfd_stage(g, 0, -, 0, U, 1, W)); with out_dev
 * non-NULL also into three caller-owned device buffers, one per component,
 * each the compact interiors (x fastest, then y, then z, storage dtype) of
 * all blocks one after the other in block order.  Any alignment works;
 * 16-byte aligned buffers move as vectors.  CFD_EINVAL if out_dev is
 * non-NULL with a NULL entry.  Asynchronous. */
cfd_status cfd_rhs_eval(cfd_grid* g, void* const out_dev[3]);

/* R = (D W)/c_dt (W ghosts must be filled), then iters weighted Jacobi
 * sweeps on P (warm start, ghosts filled) with the pressure halo refreshed
 * by each sweep, result in P.  If residual != NULL, also ||L P - R||_2 in
 * FP64 (synchronises).  Eq. 2 enforced through the pressure Poisson
 * equation. */
cfd_status cfd_pressure_solve(cfd_grid* g, double c_dt, int iters, double* residual);

/* iters weighted Jacobi sweeps on P against the current R (no divergence
 * step), ghost-on-write halo refresh, result in P.  The sweep of Sec. 4.1's
 * pressure solve on its own, e.g. to continue a solve or to time it. */
cfd_status cfd_jacobi(cfd_grid* g, int iters);

/* out = W - c_dt G P on the interior (wall-normal faces 0), ghosts of out
 * filled.  The UPDATE_VELOCITY kernel of Sec. 3 with rho = 1. */
cfd_status cfd_project(cfd_grid* g, double c_dt, int out_set);

/* One full RK2 stage (1 or 2) with time step dt, as listed above; stage 2
 * overwrites U, stage 1 writes U1. */
cfd_status cfd_rk_step(cfd_grid* g, int stage, double dt);

/* n full RK2 steps (both stages) replayed from a CUDA graph captured on the
 * first call for this dt; t += n dt.  Does not synchronise. */
cfd_status cfd_step(cfd_grid* g, double dt, int n);

/* FP64 global quantities of a velocity set over all blocks' interiors:
 * kinetic energy 1/2 sum |u|^2 hx hy hz, max |u_d|, max |D u|.  NULL
 * pointers are skipped.  Synchronises; CFD_ENONFINITE if any is NaN/Inf. */
cfd_status cfd_reduce(cfd_grid* g, int set, double* kinetic_energy, double* max_abs_u,
                      double* max_abs_div);

/* ||L P - R||_2 over all interior cells (per cell in float-float, summed in
 * FP64).  Synchronises. */
cfd_status cfd_residual(cfd_grid* g, double* residual);

/* ------------------------------------------------------------- adjoint */

/* Discrete adjoint of one RK2 step (cfd_step with n = 1) of a single
 * periodic FP32 block, order 2, ghost width 2 (the transposed advection
 * reads two cells away).  un and u1 point at element (-g,-g,-g) of three
 * arrays each, laid out like this grid's arrays (cfd_array_layout) and with
 * filled ghosts: the forward state at the start of the step and after its
 * stage-1 projection.  On entry LU, LV, LW, LP hold dL/d(u, p) after the
 * step (interior), on exit dL/d(u, p) before it.  dL/dnu of the step is
 * added to *dnu_accum_dev (device memory, one double).  Work arrays W*, U1*,
 * P, P2, R are overwritten.  Transposes: L^T = L, D^T = -G, G^T = -D; the
 * transposed Jacobi solve runs the forward sweep kernel (Sec. 4.1's
 * pressure iteration is symmetric).  CFD_EUNSUPPORTED for other grids. */
cfd_status cfd_adjoint_step(cfd_grid* g, double dt, const void* const un[3],
                            const void* const u1[3], double* dnu_accum_dev);

/* sqrt(T) checkpointed rollout for gradients of a final-time loss.
 * cfd_rollout_bytes: device bytes of the store for nsteps steps with a
 * checkpoint of (u, v, w, p) every seg steps plus seg recorded steps.
 * cfd_rollout_forward: nsteps steps from the current state (graph replay),
 * checkpointing into store.  cfd_rollout_backward: with dL/d(u_T, p_T) in
 * LU..LP, recomputes each segment from its checkpoint (last segment first),
 * recording u^n and u1 per step, and runs the adjoint steps in reverse; on
 * return LU..LP hold dL/d(u_0, p_0) and *dnu = dL/dnu (synchronises).  The
 * forward kernels are deterministic, so the recomputation reproduces the
 * forward states bitwise.  U..P are left at the end of the first segment. */
cfd_status cfd_rollout_bytes(const cfd_grid* g, int nsteps, int seg, size_t* bytes);
cfd_status cfd_rollout_forward(cfd_grid* g, double dt, int nsteps, int seg, void* store,
                               size_t bytes);
cfd_status cfd_rollout_backward(cfd_grid* g, double dt, int nsteps, int seg, void* store,
                                size_t bytes, double* dnu);

/* Simulation time and step counter (for checkpoint/resume). */
cfd_status cfd_get_state(const cfd_grid* g, double* t, long long* step);
cfd_status cfd_set_state(cfd_grid* g, double t, long long step);

/* Copy the interior of one array of one block between host memory
 * (compact (nz, ny, nx), storage dtype; pinned for asynchronous copies)
 * and the device.  to_device != 0: host -> device.  Asynchronous: the host
 * buffer must stay valid and untouched until the grid's stream has reached
 * this point.  Page-locked buffers are read or written directly by a
 * kernel over the host link (or, after cfd_set_host_copy with
 * CFD_HOST_COPY_ENGINE, by a copy engine through the staging region);
 * others go through a contiguous staging copy in the grid's memory (one
 * interior of the largest block). */
cfd_status cfd_copy_interior(cfd_grid* g, int block, int array, void* host, int to_device);

/* How cfd_copy_interior moves page-locked host memory.  CFD_HOST_COPY_KERNEL
 * (default): the pack kernel reads or writes it over the host link, one
 * pass, but its CTAs hold SMs for the whole transfer.  CFD_HOST_COPY_ENGINE:
 * a copy engine moves it to or from the staging region and the pack kernel
 * runs device to device, so a transfer on this grid's stream overlaps
 * kernels of another stream (another grid's step) with the SMs left to
 * them.  CFD_HOST_COPY_NARROW: the pack kernel reads or writes the
 * page-locked memory itself, but on one CTA per eight SMs with sixteen
 * 16-byte transfers in flight per thread, so the link stays busy while
 * another grid's step keeps the rest of the GPU (needs the block's nx a
 * multiple of 16 bytes' worth of elements and a 16-byte aligned buffer,
 * else it takes the CFD_HOST_COPY_KERNEL form).  Memory that is not
 * page-locked always takes the staging route.  CFD_EINVAL for another mode. */
typedef enum {
  CFD_HOST_COPY_KERNEL = 0,
  CFD_HOST_COPY_ENGINE = 1,
  CFD_HOST_COPY_NARROW = 2
} cfd_host_copy;
cfd_status cfd_set_host_copy(cfd_grid* g, int mode);

/* Kernel variants.  jacobi = {kind, vx, ty, zc, stages}: kind 0 is the
 * register/shuffle sweep (vx in {1,2,4} cells per thread along x, ty rows per
 * CTA in {4,8,16}), kind 1 the TMA-staged sweep (vx 4 with ty in {4,8,16}, or
 * vx 2 with ty in {8,16},
 * stages in {4,6} shared-memory planes), kind 2 the direct sweep without
 * shared memory ((vx, ty, zc) in {(4,4,1), (4,4,2), (4,4,4), (4,8,1), (4,2,4),
 * (2,4,2), (1,8,1)}, zc = z-planes per CTA), kind 3 the cp.async-staged
 * sweep (vx 4 for FP32, 8 for 16-bit storage; ty in {4,8} with stages in
 * {5,6}, or ty 2 with 6 stages), kind 5 two fused sweeps per launch (temporal blocking;
 * ty in {4,8}; used on single-block grids with nx % 128 == 0 and
 * ny % ty == 0, other grids and odd sweep counts take single sweeps),
 * kind 7 the warp-specialised TMA sweep (a producer warp fills an S-stage
 * ring, ty consumer warps; vx 4 with ty in {4,8,16} and stages in {6,8}, or
 * vx 2 (64-wide tiles, for narrow blocks) with ty in {8,16} and 6 stages),
 * kind 9 two sweeps per launch in the warp-specialised TMA form (temporal
 * blocking; vx 4 with (ty, stages) in {(16,6), (16,7), (8,5), (8,6)}, or
 * vx 2 (64-wide tiles, for narrow blocks) with ty in {8,16} and 6 stages;
 * used on single-block grids whose six faces are walls, and on grids or
 * block sets whose faces are all periodic with two ghost layers; odd sweep
 * counts and other grids take single sweeps of kind 0);
 * zc = z-planes per tile.
 * stencil = {ty in {4,8}, zc, tile_tz in {0..4}} for the point kernels:
 * rows per CTA, z chunk, and for the RHS + stage kernel either neighbour
 * reads through L1 (tile_tz 0), a z-streaming ring of shared-memory planes
 * of 32 x ty cells plus halo (tile_tz 1), the same ring 64 cells wide with
 * two x-neighbouring cells per thread in packed FP32x2 arithmetic (tile_tz
 * 3: FP32 storage and order-2 schemes, 4 rows per CTA whatever ty says;
 * elsewhere it acts as 1), or a shared-memory box of 32 x 8 x tile_tz
 * cells plus halo (2, 4).  NULL leaves a part unchanged.  Results agree
 * across variants to FP32 rounding (the same formula per cell). */
cfd_status cfd_set_kernel_config(cfd_grid* g, const int jacobi[5], const int stencil[3]);
cfd_status cfd_get_kernel_config(const cfd_grid* g, int jacobi[5], int stencil[3]);

/* Times the candidate variants on this grid (overwrites the work arrays,
 * keeps U and P) and selects the fastest; with cache_path, reuses or
 * appends a line keyed by GPU name, dtype, ghost, order and block sizes.
 * The Cactus driver's auto-tuning of the data distribution (Sec. 1.2),
 * re-targeted to the kernels' tile shapes.  Each Jacobi variant is timed
 * on runs of as many sweeps as a solve takes (rounded down to a multiple of
 * four, 4 .. 16), ghost fills between launches included.  sweep_us (may be
 * NULL) receives the chosen variant's time per sweep in microseconds. */
cfd_status cfd_autotune(cfd_grid* g, const char* cache_path, double* sweep_us);

/* Launch mode of the stencil kernels (RHS/stage, divergence, Jacobi,
 * projection) on a block set: 0 (default) = one persistent launch walks the
 * tiles of all blocks; 1 = one launch per block per kernel (the baseline the
 * batched form is measured against; its Jacobi sweeps are single sweeps,
 * so a two-sweep variant sweeps once per launch with the register kernel
 * there).  Ghost fills stay one launch.  Results are identical. */
cfd_status cfd_set_launch_mode(cfd_grid* g, int per_block);

/* Number of kernel launches this grid has enqueued so far (graph replays
 * count every kernel node once per replay). */
cfd_status cfd_stats(const cfd_grid* g, long long* kernel_launches);

/* Waits for the grid's work and reports device-side errors: CFD_ETIMEOUT
 * once any kernel has set the grid's device error flag (a bounded wait ran
 * out, or a TMA destination was misaligned).  The flag stays set, so later
 * calls keep reporting it, until memory is bound again (cfd_bind_memory /
 * cfd_alloc_memory clear it); the CUDA context stays usable.  Results
 * computed after a kernel gave up are undefined until then: such a kernel
 * leaves early, also leaving the run-time tile counter of the TMA-staged
 * sweeps off its start, which binding memory resets as well.  While the
 * flag is set, TMA-staged sweep launches (kinds 1, 7, 9) do no work, so a
 * failed solve costs one wait limit rather than one per launch. */
cfd_status cfd_check(cfd_grid* g);

/* Failure-detection self-test (the paper has no counterpart: it checks the
 * library's own device-wait bound).  Enqueues on the grid's stream one CTA
 * whose single thread initialises an mbarrier expecting one arrival and
 * waits for it through the same bounded wait the TMA-staged Jacobi kernels
 * use (form 0: the inline wait, form 1: the wait with its polling loop out
 * of line), 2 s of %globaltimer.  Nothing arrives, so the wait runs out,
 * the kernel sets the device error flag and returns; cfd_check then returns
 * CFD_ETIMEOUT.  No trap, no fault: the context and the grid's memory stay
 * usable.  Needs bound memory (CFD_ESTATE otherwise); CFD_EINVAL for
 * another form.  Asynchronous; takes about 2 s on the device. */
cfd_status cfd_selftest_wait_timeout(cfd_grid* g, int form);

/* Last error message of the calling thread (never NULL). */
const char* cfd_last_error(void);

/* ------------------------------------------------ allocation-free variant */

/* The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory when they need the diagnostics: code
 * running while its stream is being captured into a CUDA graph (cudaMalloc
 * is not capturable), host frameworks whose device memory belongs to their
 * own pool allocator, and hooks inside a time loop that must not pay the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 *
 * Same quantities as cfd_reduce, from raw device pointers, allocating
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine):
 * u, v, w point at interior element (0,0,0) of three arrays of storage dtype
 * `dtype` (cfd_dtype) with row pitch pitch_y and plane pitch pitch_z
 * (elements); the elements at index -1 along x (u), y (v) and z (w) must be
 * readable (the divergence reads them).  dims = interior (nx, ny, nz),
 * h = cell size.  out_dev is caller-owned device memory for 4 doubles:
 * {1/2 sum |u|^2 hx hy hz, max |u_d|, max |D u|, number of non-finite
 * values}, written asynchronously on `stream` (a cudaStream_t, may be NULL).
 *
 * Scratch: per-plane partial sums live in one file-scope static device
 * array of the library, 4096 planes x 4 doubles (128 KiB), which every GPU
 * that loads the library keeps until process exit.  nz > 4096 returns
 * CFD_EINVAL.  All calls share that array and it keeps the last call's
 * contents (each call overwrites every slot it later reads, so nothing needs
 * clearing); calls that overlap on the GPU (different streams, or several
 * host threads) race on it and must be serialised by the caller.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Errors: CFD_EINVAL for bad sizes or pointers, CFD_ECUDA if the launch
 * fails; the message is in cfd_noalloc_last_error(). */
cfd_status cfd_reduce_velocity_noalloc(const void* u, const void* v, const void* w, int dtype,
                                       const int dims[3], long long pitch_y, long long pitch_z,
                                       const double h[3], double* out_dev, void* stream);

/* Last error message of cfd_reduce_velocity_noalloc on this thread. */
const char* cfd_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
