/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for the
 * volume-averaged Navier-Stokes equations (VANSE) with Carreau-Yasuda blood
 * rheology and a coil represented as a porous medium, after
 * M. Horvat, S. B. Lunowa, D. Sytnyk, B. Wohlmuth, "A Lattice Boltzmann Method
 * for Non-Newtonian Blood Flow in Coiled Intracranial Aneurysms",
 * arXiv 2402.10809 (the "paper" below).
 *
 * Conventions shared by every call
 *  - Grid arrays are dense, x fastest: cell index = x + nx * (y + ny * z).
 *  - Lattice units inside: dx = dt = 1, c_s^2 = 1/3; physical parameters are
 *    converted with the spacing, time step and reference density of Table 1.
 *  - Memory: the library never allocates device memory.  The caller passes one
 *    device workspace of at least lbm_workspace_size() bytes, 256-byte
 *    aligned, and keeps it alive until lbm_destroy().  The context itself is a
 *    small host object.  All work is enqueued on the caller's CUDA stream;
 *    calls that return host data synchronise that stream.
 *  - Errors: every call returns an lbm_status; lbm_last_error() gives a text.
 *    No call aborts, traps or asserts on the device.
 *  - One context serves one stream; calls on one context must not overlap.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* bad argument, size or geometry */
    LBM_ENOMEM = 2,    /* workspace or destination too small */
    LBM_ECUDA = 3,     /* a CUDA runtime call failed (text in lbm_last_error) */
    LBM_EUNSTABLE = 4, /* non-finite state detected by the periodic check */
    LBM_ESTATE = 5     /* call not valid in the current state */
} lbm_status;

/* Cell flags (uint8). */
enum { LBM_SOLID = 0, LBM_FLUID = 1, LBM_INLET = 2, LBM_OUTLET = 3 };

/* Storage of the particle densities f_i in HBM.  All arithmetic is FP32.
 * F32:      f_i - w_i phi_hat stored as float;
 * F16DEV:   the same deviation stored as IEEE binary16 (round to nearest even);
 * BF16DEV:  the same deviation stored as bfloat16 (round to nearest even).
 * phi_hat is the porosity of the cell the value streams to (the cell's own
 * porosity where that neighbour is solid or outside), so a value is always
 * decoded with the porosity of the cell that reads it. */
enum { LBM_F32 = 0, LBM_F16DEV = 1, LBM_BF16DEV = 2 };

typedef struct {
    int32_t nx, ny, nz;    /* box size, each 2..1024 */
    int32_t q;             /* velocity set: 27 (the paper's D3Q27, Sec. 3) or 19 */
    int32_t storage;       /* LBM_F32, LBM_F16DEV or LBM_BF16DEV */
    int32_t periodic[3];   /* 1: axis wraps around */
} lbm_grid;

/* Carreau-Yasuda law, Eq. (3): mu(g) = mu_inf + (mu0 - mu_inf)(1 + (lambda g)^a)^((n-1)/a),
 * in SI units; rho0 [kg/m^3], dx [m], dt [s] map them to the lattice (Table 1):
 * nu_lattice = mu / rho0 * dt / dx^2, lambda_lattice = lambda / dt.
 * Pass rho0 = dx = dt = 1 to give lattice values directly. */
typedef struct {
    double mu0, mu_inf, lambda, n, a;
    double rho0, dx, dt;
} lbm_rheology;

/* Darcy-Forchheimer drag of Sec. 2, f(u) = -phi^2 nu u / k - phi^3 C_F |u| u / sqrt(k),
 * with Kozeny-Carman k = phi^3 d_p^2 / (150 (1 - phi)^2) and Ergun
 * C_F = 1.75 / sqrt(150 phi^3).  d_p [m]; k_const [m^2] > 0 replaces
 * Kozeny-Carman by a constant permeability (acting where phi < 1);
 * nu_darcy [m^2/s] <= 0 selects nu = mu0 / rho0 (Sec. 4); forchheimer 0/1. */
typedef struct {
    double d_p, k_const, nu_darcy;
    int32_t forchheimer;
} lbm_porous;

/* Forcing and open boundaries (Sec. 4).  body_force: per unit mass, lattice units.
 * Inlet (Zou-He velocity inlet): cells flagged LBM_INLET on the face
 * inlet_axis (0 x, 1 y, 2 z), inlet_side (0 low, 1 high); Hagen-Poiseuille
 * profile u_perp = 2 v(t) max(0, 1 - r^2 / R^2) with r measured from
 * inlet_center (lattice coordinates, cell centres at integer + 1/2) and
 * R = inlet_radius; mean velocity v(t) = u0 (1 + amp sin(2 pi t / period)),
 * ramped linearly over the first ramp_steps steps when ramp_steps > 0.
 * Outlet: cells flagged LBM_OUTLET on the face outlet_axis / outlet_side,
 * non-equilibrium extrapolation from the first interior neighbour with the
 * prescribed density rho_out.  An axis of -1 disables that boundary. */
typedef struct {
    double body_force[3];
    int32_t inlet_axis, inlet_side;
    double inlet_center[3];
    double inlet_radius, u0, amp, period, ramp_steps;
    int32_t outlet_axis, outlet_side;
    double rho_out;
} lbm_bc;

/* Length of the packed layout for these flags (host memory): the library
 * stores, for every x-row (y, z) of the box, the span from the first to the
 * last non-solid cell of that row, and packs these spans back to back; the
 * result is the sum of the span lengths (non-solid cells plus the solid cells
 * inside spans).  -1 on bad input. */
int64_t lbm_list_length(const lbm_grid* grid, const uint8_t* flags);

/* Bytes of device workspace for a packed layout of n_list slots (from
 * lbm_list_length; pass n_list < 0 for the bound nx*ny*nz).  The distribution
 * buffers take 2 Q n_list elements; the rest is per-box (flags, porosity,
 * region: 6 bytes per box cell) and per-row.  0 on a bad grid. */
size_t lbm_workspace_size(const lbm_grid* grid, int64_t n_list);

/* Creates a context and sets the initial state (Sec. 3, Sec. 4):
 * f_i = f_i^eq(rho = 1, u = 0) = w_i phi, omega = omega(mu0) at rho = 1, and
 * the inlet / outlet reconstruction of time 0 is applied by the first step.
 *  flags     [nz][ny][nx] uint8 LBM_SOLID / FLUID / INLET / OUTLET;
 *  porosity  [nz][ny][nx] float, phi in (0, 1]; phi must be 1 on inlet and
 *            outlet cells and on each outlet cell's interior neighbour, which
 *            must be LBM_FLUID;
 *  inputs_on_device: 1 if flags / porosity are device pointers, 0 for host;
 *  workspace / workspace_bytes: caller-owned device memory (see above);
 *  stream: a cudaStream_t (NULL = legacy default stream).
 * The inputs are copied into the workspace; the caller may free them after
 * this call returns.  Returns LBM_EINVAL on bad sizes, flags or porosity. */
lbm_status lbm_init(lbm_ctx** ctx, const lbm_grid* grid, const uint8_t* flags, const float* porosity,
                    int32_t inputs_on_device, const lbm_rheology* rheology, const lbm_porous* porous,
                    const lbm_bc* bc, void* workspace, size_t workspace_bytes, void* stream);

/* Advances n >= 0 time steps (Sec. 3): each step pulls f(t) from the neighbours
 * (half-way bounce-back at walls, Zou-He inlet, extrapolation outlet), computes
 * rho, u (explicit Darcy-Forchheimer velocity), the force, Pi, the shear rate
 * gdot = omega(t-1) ||Pi||_F / (c_s^2 rho), mu(gdot) and omega(t), collides
 * with Omega^phi + Omega^f + Omega^SRT and stores f*(t).  Asynchronous. */
lbm_status lbm_step(lbm_ctx* ctx, int32_t n);

/* Fields of the current time t on the dense box (0 at solid cells):
 * rho [N], u [3][N] (x, y, z planes), shear_rate gdot(t) [N], omega(t) [N].
 * Any pointer may be NULL.  dst_on_device: 1 device pointers (asynchronous),
 * 0 host pointers (synchronises the stream). */
lbm_status lbm_moments(lbm_ctx* ctx, float* rho, float* u, float* shear_rate, float* omega,
                       int32_t dst_on_device);

/* Diagnostics of the current time, accumulated in FP64 (sac averages of the
 * paper's Sec. 4 results among them): out[0] mass sum_x sum_i f_i,
 * out[1] kinetic energy sum rho |u|^2 / 2, out[2] sum of |u| over the region,
 * out[3] number of region cells, out[4] max |u|, out[5] min omega,
 * out[6] max omega, out[7] number of non-finite cells.  region: [N] uint8
 * (nonzero = in the region) or NULL for an empty region; region_on_device
 * tells where it lives.  out is host memory; the call synchronises. */
lbm_status lbm_diag(lbm_ctx* ctx, const uint8_t* region, int32_t region_on_device, double out[8]);

/* Wall-shear-stress proxy of the current time t on the dense box (the
 * quantity whose sac-wall average the paper reports beside the velocity,
 * Sec. 4 results: tau = sigma n - (n . sigma n) n).  Voxel form: at a fluid
 * cell with links to the wall (neighbours that are solid or outside the box),
 * n is the normalised sum of w_i c_i over those links, sigma = -(1 - omega/2) Pi
 * the viscous stress from the corrected second moment Pi of the shear rate,
 * with omega the rate of the collision of time t.  wss [N] receives |tau| in
 * lattice units (multiply by rho0 dx^2 / dt^2 for Pa); 0 on cells without wall
 * links, on inlet / outlet cells and on solid cells.  dst_on_device: 1 device
 * pointer (asynchronous), 0 host pointer (synchronises). */
lbm_status lbm_wall_shear(lbm_ctx* ctx, float* wss, int32_t dst_on_device);

/* lbm_diag without caller scratch (the paper has no counterpart; this is a
 * deployment convenience).  Same outputs as lbm_diag, computed by the same
 * kernels, but the per-block partial sums and the device-side result live in a
 * fixed array inside the library instead of the caller's workspace, and the
 * call allocates nothing.  It is meant for callers that may not allocate
 * device memory where they need the diagnostics, e.g. a monitoring thread of a
 * host application whose device allocator is owned by another framework.
 *  - Limit: at most 8,388,608 slots of the packed layout (lbm_list_length)
 *    and a diagnostics launch of at most 98,305 blocks, which holds any
 *    context with up to 1,048,576 cells on periodic faces, inlet or outlet
 *    (LBM_EINVAL beyond, with the block count in the message; use lbm_diag);
 *    the array costs every GPU that loads the library 6.75 MiB until exit.
 *  - region: device memory of the current device, or NULL (host regions are
 *    rejected with LBM_EINVAL, since copying them would need scratch; so is
 *    device memory of another GPU); out: host memory; synchronises.
 *  - The context's device must be current (its workspace may also be managed
 *    memory).  Every call outside stream capture looks up the array's device
 *    address (cudaGetSymbolAddress), so a device reset followed by a new
 *    context is safe; a call during capture reuses the last address looked up
 *    on that device, so make the first call on a device before any capture.
 *  - All calls share the array: calls that overlap on the GPU race; serialise
 *    them.  No state carries over from one call to the next. */
lbm_status lbm_diag_noalloc(lbm_ctx* ctx, const uint8_t* region, double out[8]);

/* Anisotropic permeability (Sec. 3 remark on the velocity solution).  The
 * drag becomes f(u) = -phi^2 nu K^{-1} u - phi^3 C_F |u| K^{-1/2} u with
 * K = k(phi) S^{-1}: k(phi) and C_F the isotropic closure of lbm_init
 * (Kozeny-Carman or constant permeability, Ergun's C_F; nu the Darcy
 * viscosity) and S a symmetric positive definite shape tensor per cell
 * (S = Id is the isotropic medium).  Every later step, moments, diag and
 * wall-shear call solves the velocity equation (A + |u| B) u = v,
 * A = Id + (phi nu / 2) K^{-1}, B = (phi^2 C_F / 2) K^{-1/2}, at each cell with
 * phi < 1 by the fixed-point iteration u_{m+1} = (A + |u_m| B)^{-1} v from
 * u_0 = v, until |u_{m+1} - u_m| <= tol |v| or max_iter iterations (FP32);
 * cells with phi = 1 keep the explicit solution.
 *  - shape:  [6][nz][ny][nx] float, components xx yy zz xy xz yz (each a
 *            dense plane); device memory; read only during the call.  NULL
 *            switches back to the isotropic closure.
 *  - buffer / bytes: caller-owned device memory (256-byte aligned) of at least
 *            lbm_anisotropy_buffer_size(ctx) bytes (12 floats per slot of the
 *            packed layout) that the context keeps using until the next
 *            lbm_set_anisotropy or lbm_destroy.  The set-up stores A - Id and
 *            B per slot there, with S^{1/2} from an FP64 Jacobi
 *            eigendecomposition.
 *  - max_iter 1..1000, 0 <= tol < 1 (1e-6 and 16 converge to FP32 round-off
 *            for blood-flow drag).
 * Any storage type.  LBM_EINVAL when S is not finite
 * or not positive definite at a cell with phi < 1; LBM_ENOMEM when the buffer
 * is too small.  lbm_adjoint differentiates the anisotropic solve too (the
 * implicit-function reverse of its converged velocity, with the porosity
 * dependence of the closure; S itself is held fixed): its gradient is that of
 * the converged solve, so give max_iter and tol that converge (the defaults
 * do); with a truncated iteration the gradient no longer belongs to the
 * computed objective.  Synchronises the stream. */
size_t lbm_anisotropy_buffer_size(const lbm_ctx* ctx);
lbm_status lbm_set_anisotropy(lbm_ctx* ctx, const float* shape, void* buffer, size_t bytes, int32_t max_iter,
                              float tol);

/* z-slab decomposition of one problem over several contexts (one per GPU, or
 * several on one device): the partition the fused step admits (Sec. 3: a cell
 * pulls only from its 26 neighbours, so a slab of z-planes needs one plane of
 * its neighbours per face and, across a face, only the 9 (D3Q27) or 5 (D3Q19)
 * populations whose c_z points into the slab).  The paper runs one GPU; this
 * is the sharding of a box too large for one.  A slab owns z in [z0, z1) of
 * the box and is set up with lbm_init on the sub-box [z0 - h0, z1 + h1) of the
 * box's flags and porosity, h0 = 1 if it has a lower neighbour (z0 > 0), h1 = 1
 * if it has an upper one, and the box's other parameters unchanged (the inlet
 * and outlet stay where they are: only the slab that holds their cells sees
 * them).  Boxes periodic in z are not sharded.
 *
 * lbm_slab_bounds: z0 of every slab and the box's nz in z_bounds[0..nslabs],
 *   chosen so that the slabs hold about equal numbers of packed slots, every
 *   slab at least one plane; host only (no device, no context).
 * lbm_plane_slots: first slot and number of slots of z-plane z in the packed
 *   layout of (grid, flags) (planes are contiguous ranges); host only.
 * lbm_set_halo: marks the first lo_planes and last hi_planes (0 or 1 each)
 *   z-planes of the context as halo planes: lbm_step neither updates them nor
 *   do lbm_moments (zeros there) and lbm_diag count them; their populations
 *   come from the neighbours (their slots become ghost slots without stores;
 *   calling it again restores the previous halo planes first).  LBM_EINVAL
 *   for other counts, for no interior plane left, or for a box periodic in z;
 *   lbm_adjoint refuses a context with halo planes (the adjoint runs on one
 *   domain).  Synchronises the stream.
 * lbm_halo_message_size: bytes a face sends (side 0 the lower face, 1 the
 *   upper face): the populations of the interior plane next to the face whose
 *   c_z points through it, [directions in increasing index][plane slots] in
 *   the storage type; 0 without a halo on that side.
 * lbm_halo_pack / lbm_halo_unpack: device buffers of that layout; pack reads
 *   the interior plane next to the face, unpack writes the halo plane of the
 *   face (the message the neighbour packed on its side facing this one: side 1
 *   of the lower slab pairs with side 0 of the upper slab).  Asynchronous on
 *   the context's stream.
 * lbm_halo_exchange: both copies of one face between two contexts on one
 *   device in one launch (lower's top interior plane to upper's lower halo,
 *   upper's first interior plane to lower's upper halo); the two contexts must
 *   share one stream.  LBM_EINVAL when the face's planes do not match.
 * One time step of the sharded problem: lbm_step(ctx, 1) on every slab, then
 * every face exchanged (or packed, sent, received and unpacked).  Every cell's
 * arithmetic is then the same as in the unsharded box, so the results are
 * bit-identical to it; the diagnostics of the box are the sums (mass, kinetic
 * energy, region sums, non-finite count) and extrema of the slabs'. */
lbm_status lbm_slab_bounds(const lbm_grid* grid, const uint8_t* flags, int32_t nslabs, int32_t* z_bounds);
lbm_status lbm_plane_slots(const lbm_grid* grid, const uint8_t* flags, int32_t z, int64_t* first, int64_t* count);
lbm_status lbm_set_halo(lbm_ctx* ctx, int32_t lo_planes, int32_t hi_planes);
size_t lbm_halo_message_size(const lbm_ctx* ctx, int32_t side);
lbm_status lbm_halo_pack(lbm_ctx* ctx, int32_t side, void* dst);
lbm_status lbm_halo_unpack(lbm_ctx* ctx, int32_t side, const void* src);
lbm_status lbm_halo_exchange(lbm_ctx* lower, lbm_ctx* upper);

/* lbm_step_slabs: `steps` time steps of the n adjacent z-slabs slabs[0..n-1]
 * (bottom to top) of one problem on one device, each slab on its own
 * context's stream (the streams may differ or coincide): every slab's step
 * waits only for the exchanges of its own faces, and each face's exchange
 * (as lbm_halo_exchange, launched on the lower slab's stream) only for the
 * steps of its two slabs, so slabs step concurrently.  join_stream (NULL:
 * the default stream) orders the whole run after its earlier work and its
 * later work after the run.  The same results as lbm_step of every slab followed by
 * lbm_halo_exchange of every face, step by step.  Returns the first error;
 * LBM_EINVAL for slabs that are not adjacent slabs of one lattice. */
lbm_status lbm_step_slabs(lbm_ctx** slabs, int32_t n, int32_t steps, void* join_stream);

/* Volume-averaged porosity of a voxelised coil, the input that lbm_init takes
 * as the porosity of the averaged simulations (Sec. 4: the porosity field is
 * the windowed convolution of the voxelised coil with a uniform averaging
 * kernel; Table 1: averaging window 1.23 mm).  No context is involved: this
 * runs before lbm_init.  For every cell x of the nx * ny * nz box:
 *     count(x) = number of wire voxels v with x_a - lo <= v_a <= x_a + hi on
 *                every axis a, lo = window / 2, hi = window - 1 - lo (cells
 *                outside the box hold no wire);
 *     phi(x)   = max(phi_min, (window^3 - count(x)) / window^3), the quotient
 *                correctly rounded to FP32 (count and window^3 are exact
 *                integers), and phi(x) = 1 where flags[x] == LBM_SOLID.
 *  - wire:  [nz][ny][nx] uint8, nonzero = wire voxel; device memory.
 *  - flags: [nz][ny][nx] uint8 (the flags of lbm_init) or NULL for no solid
 *           override; device memory.
 *  - phi:   [nz][ny][nx] float, written; device memory.
 *  - workspace: caller-owned device scratch, 256-byte aligned, at least
 *           lbm_porosity_workspace_size(nx, ny, nz) bytes (3 bytes per cell).
 *  - cuda_stream: the stream the three passes run on (asynchronous).
 * Limits: 1 <= nx <= 16384, window 1..255 (window^2 fits the 16-bit
 * intermediate, window^3 < 2^24), 0 <= phi_min <= 1.  Returns LBM_EINVAL on
 * bad sizes, window, phi_min, pointers or alignment, LBM_ENOMEM when the
 * workspace is too small, LBM_ECUDA when a launch fails (there is no context,
 * hence no lbm_last_error text).  lbm_porosity_workspace_size returns 0 for
 * bad sizes. */
size_t lbm_porosity_workspace_size(int32_t nx, int32_t ny, int32_t nz);
lbm_status lbm_porosity_average(int32_t nx, int32_t ny, int32_t nz, const uint8_t* wire, const uint8_t* flags,
                                int32_t window, float phi_min, float* phi, void* workspace, size_t workspace_bytes,
                                void* cuda_stream);

/* L2 residency of the time step (no counterpart in the paper; a property of
 * the GPU execution).  Every step reads the per-slot words (row id, link mask,
 * omega, porosity: 16 bytes per slot) while the populations stream past them.
 * lbm_init keeps up to a quarter of the L2 cache's worth of them in its
 * persisting part through an access-policy window on the step and reverse-
 * step launches, raising the process's CUDA limit
 * cudaLimitPersistingL2CacheSize to hold the window (never lowering it; a
 * limit of the process's context, gone when the process exits).  lbm_step
 * and lbm_adjoint of a context first return the persisting lines of the
 * context that used them before to normal (cudaCtxResetPersistingL2Cache), and
 * lbm_destroy those of its own, so contexts do not crowd each other out.
 *  - lbm_set_l2_window: max_bytes < 0 the default (a quarter of the L2),
 *    0 no window, > 0 at most that many bytes.  Results are identical either
 *    way.
 *  - lbm_l2_window_bytes: the window in bytes (0 none; -1 bad context).
 *  - lbm_set_l2_group: contexts given the same nonzero group (the z-slabs of
 *    one problem stepping in turn on one device) take the persisting L2 over
 *    from each other without returning the other's lines to normal; their
 *    windows should fit the L2's persisting part together.  0 (the default)
 *    leaves a context on its own. */
lbm_status lbm_set_l2_window(lbm_ctx* ctx, int64_t max_bytes);
int64_t lbm_l2_window_bytes(const lbm_ctx* ctx);
lbm_status lbm_set_l2_group(lbm_ctx* ctx, int64_t group);

/* Every check_every steps of later lbm_step calls, run the non-finite count of
 * lbm_diag and return LBM_EUNSTABLE when it is nonzero (0 = never, default). */
lbm_status lbm_set_check(lbm_ctx* ctx, int32_t check_every);

/* Discrete adjoint (reverse mode of the time step of lbm_step) for gradients
 * of a sac flow quantity with respect to the porosity field phi, the coil
 * distribution of Sec. 2 (the paper itself runs forward simulations only; the
 * objective below is its sac-averaged flow quantity of Sec. 4 made a scalar):
 *     J = (1/T) sum_{t=1..T} (1/|R|) sum_{y in R} rho(t, y) |u(t, y)|^2 / 2,
 * R = non-solid cells whose region byte is nonzero, rho and u as in the
 * collision of time t.  The call restarts from the rest state of lbm_init
 * (t = 0), runs T forward steps keeping a checkpoint every K steps, then sweeps
 * backwards, replaying one segment of K steps at a time from its checkpoint.
 * The context's own state and time are left untouched.
 *
 * lbm_adjoint_workspace_size: bytes of device workspace for (T, K); 0 on an
 *   invalid context or T < 1 or K < 1.  About (ceil(T/K) + min(K, T)) states
 *   in the storage type plus min(K, T) dense FP32 density fields plus two FP32
 *   adjoint states.  K >= T keeps the whole trajectory (no replay).
 * lbm_adjoint:
 *   objective 0: the kinetic-energy objective above; 1: the same time mean of
 *            the wall-shear-stress proxy |tau| of lbm_wall_shear, averaged over
 *            the cells of R with wall links (the sac-wall average of Sec. 4);
 *   region   [N] uint8, host or device memory (region_on_device);
 *   workspace / workspace_bytes: caller-owned device memory, 256-byte aligned;
 *   grad     [N] FP64 device memory, overwritten with dJ/dphi (0 on solid
 *            cells); the accumulation over time steps is in FP64;
 *   J        host double, the objective value.
 * Synchronises the context's stream.  LBM_EINVAL on bad arguments or a region
 * without fluid cells (for objective 1: without wall cells), LBM_ENOMEM when
 * the workspace is too small. */
size_t lbm_adjoint_workspace_size(const lbm_ctx* ctx, int32_t T, int32_t K);
lbm_status lbm_adjoint(lbm_ctx* ctx, int32_t T, int32_t K, int32_t objective, const uint8_t* region,
                       int32_t region_on_device, void* workspace, size_t workspace_bytes, double* grad, double* J);

/* Checkpoint of the full state (distributions, relaxation rates, time): size in
 * bytes, save into / load from caller memory (host or device). */
size_t lbm_state_size(const lbm_ctx* ctx);
lbm_status lbm_save(lbm_ctx* ctx, void* dst, size_t bytes, int32_t dst_on_device);
lbm_status lbm_load(lbm_ctx* ctx, const void* src, size_t bytes, int32_t src_on_device);

/* Current time step, number of non-solid cells, and the last error text. */
int64_t lbm_time(const lbm_ctx* ctx);
int64_t lbm_fluid_count(const lbm_ctx* ctx);
const char* lbm_last_error(const lbm_ctx* ctx);

/* Releases the host context (the workspace stays the caller's). */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
