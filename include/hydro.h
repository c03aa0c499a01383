/*
 * hydro.h -- C ABI of the GB300 hydro library (libhydro_gb300.so).
 *
 * The library advances boxes of the 3D compressible Euler equations for an
 * ideal gamma-law gas by unsplit PPM Godunov steps: conserved-to-primitive
 * conversion, PPM reconstruction with monotonicity limiters and shock
 * flattening, characteristic tracing to half-step face states, 3D
 * corner-transport-upwind (CTU) transverse corrections, HLLC Riemann solves,
 * the conservative flux-divergence update and the CFL time-step reduction.
 *
 * Source of the operations.  The paper (Katz et al., "Preparing Nuclear
 * Astrophysics for Exascale") states the problem: data lives in boxes
 * ("Fabs") bounded by lo/hi indices with several components (§2, Fig. 1),
 * is kept resident on the GPU for the whole run (§3, memory management),
 * and is advanced by a stencil that computes limited slopes from
 * neighbouring zones and reconstructs a polynomial of the fluid state (§3);
 * throughput is reported as zones updated per unit time (§4).  The numerical
 * method itself is the published PPM/CTU/HLLC family the paper's code uses
 * (Colella & Woodward 1984; Colella 1990; Saltzman 1994; Toro, Spruce &
 * Speares 1994).
 *
 * Conventions shared by every call:
 *  - Pointers named *_dev are CUDA device pointers on the current device;
 *    pointers named *_host are host pointers (pinned memory gives the best
 *    copy speed but is not required).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns an int status: HYDRO_OK (0), HYDRO_PENDING (> 0, poll
 *    only) or a negative HYDRO_ERR_* code.  hydro_last_error() returns a
 *    thread-local message describing the last failure.  No exception crosses
 *    the ABI.
 *  - Launching calls are asynchronous: device-side errors (a nonphysical state
 *    after an update) are reported by the next hydro_sync().
 *  - The library never allocates device memory: the caller passes the state
 *    and scratch buffers (sized by hydro_workspace_size) and keeps ownership.
 */
#ifndef HYDRO_GB300_H
#define HYDRO_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HYDRO_OK 0
#define HYDRO_PENDING 1
#define HYDRO_ERR_INVALID (-1)     /* bad argument or descriptor */
#define HYDRO_ERR_NOMEM (-2)       /* buffer too small or over the memory budget */
#define HYDRO_ERR_NONPHYSICAL (-3) /* rho <= 0, p <= 0 or NaN after an update */
#define HYDRO_ERR_TIMEOUT (-4)     /* a bounded device wait of the persistent form gave up */
#define HYDRO_ERR_CUDA (-5)        /* a CUDA runtime call failed */

/* ---- boundary conditions (one per box face) ---- */
#define HYDRO_BC_PERIODIC 0 /* copy from the opposite side; must be set on both faces of an axis */
#define HYDRO_BC_OUTFLOW 1  /* zero-gradient copy of the last interior zone */
#define HYDRO_BC_REFLECT 2  /* mirror image, normal momentum negated */

/* ---- precision of the reconstruction/Riemann stages ---- */
#define HYDRO_FP64 0  /* every stage in FP64 */
#define HYDRO_MIXED 1 /* FP32 flattening, reconstruction, tracing, CTU corrections and Riemann
                         solves (FP32 scratch fields); FP64 state, primitive conversion, dt
                         reduction and flux-divergence update, so each face flux is applied to
                         both neighbours in FP64 and conservation holds to FP64 round-off */

#define HYDRO_NG 4 /* ghost zones per side (the only supported value) */

/* One box.  Zones are (i,j,k) with i in [0,nx) interior and [-ng, nx+ng) with ghosts. */
typedef struct hydro_box_desc {
  int32_t nx, ny, nz; /* interior zones per axis, each >= 4 */
  int32_t ng;         /* ghost zones per side: HYDRO_NG */
  double dx, dy, dz;  /* zone widths, > 0 */
  double gamma;       /* ratio of specific heats, > 1 */
  double cfl;         /* Courant number, in (0, 1] */
  int32_t bc[6];      /* HYDRO_BC_* for faces xlo, xhi, ylo, yhi, zlo, zhi */
  int32_t precision;  /* HYDRO_FP64 or HYDRO_MIXED; boxes of one handle may differ */
} hydro_box_desc;

/* Where box `box` lives inside the state buffer, in FP64 elements.
 * Conserved variable v (0 rho, 1 rho*u, 2 rho*v, 3 rho*w, 4 E) of zone (i,j,k),
 * ghosts included, is element
 *   offset + v*var_stride + (k+ng)*plane + (j+ng)*pitch + (i+ng).        */
typedef struct hydro_layout {
  int64_t offset;     /* first element of the box */
  int64_t pitch;      /* elements between rows: nx+2ng rounded up to a multiple of 4 */
  int64_t plane;      /* elements between planes: pitch*(ny+2ng) */
  int64_t var_stride; /* elements between variables: plane*(nz+2ng) rounded up to 32 */
} hydro_layout;

typedef struct hydro_handle hydro_handle;

/* Bytes of device memory needed for `nboxes` boxes described by d[0..nboxes-1]:
 * the FP64 state (all boxes, ghosts included) and the scratch space (face
 * states, fluxes, per-box time-step data).  Returns HYDRO_ERR_INVALID for a bad
 * descriptor (the message names the box and field). */
int hydro_workspace_size(const hydro_box_desc* d, int nboxes, size_t* state_bytes,
                         size_t* scratch_bytes);

/* Layout of box `box` in the state buffer (see hydro_layout). */
int hydro_box_layout(const hydro_box_desc* d, int nboxes, int box, hydro_layout* out);

/* Creates a handle over caller-owned device buffers of at least the sizes
 * given by hydro_workspace_size.  Source: the paper's boxes of data ("Fabs")
 * with lo/hi bounds and several components (§2, Fig. 1), kept resident on the
 * GPU for the whole run (§3, memory management).  state_dev and scratch_dev
 * must be 256-byte aligned and stay valid until hydro_free (the library
 * borrows them and never frees them).  Copies the box table into the head of
 * scratch_dev (synchronously) and zeroes the per-box time, dt and status.  The
 * state contents are left alone.  *out receives the handle.  Errors:
 * HYDRO_ERR_INVALID (bad descriptor, null or misaligned buffer; *out stays
 * NULL), HYDRO_ERR_NOMEM (a buffer smaller than hydro_workspace_size asks),
 * HYDRO_ERR_CUDA. */
int hydro_alloc(const hydro_box_desc* d, int nboxes, void* state_dev, size_t state_bytes,
                void* scratch_dev, size_t scratch_bytes, hydro_handle** out);

/* Releases the handle (host memory only; the caller frees the buffers). */
int hydro_free(hydro_handle* h);

/* Fills the ghost zones of every box from its boundary conditions, in the
 * order x, then y, then z, so that edges and corners are filled too.  Source:
 * the ghost cells around each box's lo/hi interior that the stencil reads
 * (§2, Fig. 1; §3).  Asynchronous on `stream`; HYDRO_ERR_INVALID for a null
 * handle or one used on another device, HYDRO_ERR_CUDA on a launch failure. */
int hydro_fill_ghosts(hydro_handle* h, void* stream);

/* Computes each box's CFL time step from its current interior state,
 * dt_b = cfl / max over zones and axes of (|u_a| + c) / dx_a (the CFL step
 * cfl * min dx_a / (|u_a| + c)), into dt_dev[0..nboxes-1] (device memory,
 * caller-owned, written asynchronously).  Source: the time step set by the
 * zone width and the signal speed, which makes the paper's throughput a count
 * of zones per time step (§4).  The ghost zones must be filled (the
 * primitive conversion runs over the ghosted box).  Errors as for
 * hydro_fill_ghosts. */
int hydro_compute_dt(hydro_handle* h, double* dt_dev, void* stream);

/* Advances every box by `nsteps` steps.  Each step fills the ghost zones,
 * takes dt from dt_dev[b] (or, if dt_dev is NULL, computes it from the state
 * as hydro_compute_dt does) and applies one unsplit PPM/CTU/HLLC update to the
 * interior.  Source: the hydro update of §3 (limited slopes from neighbouring
 * zones, a reconstructed polynomial, fluxes, the state update), applied to
 * every zone of every box per step as the paper's zones-per-time-step
 * throughput counts it (§4).  nsteps == 0 does nothing.  Asynchronous on
 * `stream`; device-side errors (a nonphysical state, a persistent-form
 * timeout) are reported by the next hydro_sync.  HYDRO_ERR_INVALID for a null
 * handle or nsteps < 0, HYDRO_ERR_CUDA on a launch failure. */
int hydro_step(hydro_handle* h, const double* dt_dev, int nsteps, void* stream);

/* Waits for `stream`, then reports the first device-side error:
 * HYDRO_ERR_TIMEOUT if a wait of the persistent form gave up (the interrupted
 * step is incomplete; the per-box signal-speed maxima are cleared so that the
 * next step starts clean), else HYDRO_ERR_NONPHYSICAL if an update produced
 * rho <= 0, p <= 0 or NaN in some box.  The error flags are cleared after
 * being reported. */
int hydro_sync(hydro_handle* h, void* stream);

/* Simulated time advanced so far by each box, into time_host[0..nboxes-1]
 * (synchronous on `stream`). */
int hydro_get_time(hydro_handle* h, double* time_host, void* stream);

/* Copies interior states between host memory and the device state.
 * The host array is [box][v][k][j][i] over interior zones only, boxes in
 * order, FP64, exactly sum_b 5*nx*ny*nz*8 bytes (`bytes` must match).  The
 * copy goes through the scratch space (which it overwrites) and a gather/
 * scatter kernel; both calls return once the host buffer may be reused. */
int hydro_upload(hydro_handle* h, const double* state_host, size_t bytes, void* stream);
int hydro_download(hydro_handle* h, double* state_host, size_t bytes, void* stream);

/* Diagnostics: where the per-zone intermediates of box `box` live inside the
 * scratch buffer, for stage-by-stage checks.  *offset_bytes receives the byte
 * offset of the box's first field from the start of scratch_dev, *nfields the
 * number of fields (138) and *elem_bytes their element size (8 for
 * HYDRO_FP64, 4 for HYDRO_MIXED boxes).  Each field is a ghosted-box grid with
 * the state's pitch, plane and var_stride (in elements; fields are var_stride
 * elements apart), in this order: primitive q[5] = (rho,u,v,w,p); sound speed
 * c; flattening coefficient chi; left-edge states qm[3][5] and right-edge
 * states qp[3][5] per axis d in the normal frame of d (rho, u_d, u_{d+1},
 * u_{d+2}, p, axis indices mod 3); normal fluxes f0[3][5]; once-corrected
 * fluxes f1[6][5] for the ordered axis pairs xy,xz,yx,yz,zx,zy; final fluxes
 * f[3][5]; limited slopes dq[3][5] of the normal-frame variables of each axis;
 * conserved momenta (normal frame) and total energy of the left- and right-edge
 * states, um[3][4] and up[3][4], then 1/c and c/rho of each zone (these ten
 * for HYDRO_FP64 boxes only: HYDRO_MIXED boxes form them where they are
 * needed).
 * Fluxes are conserved-variable components; the flux through the low face of
 * zone (i,j,k) along d is stored at (i,j,k).  Values are defined only where
 * the step computes them (see also hydro_fuse_lines and hydro_set_method for
 * what dq holds). */
int hydro_debug_fields(const hydro_box_desc* d, int nboxes, int box, int64_t* offset_bytes, int32_t* nfields,
                       int32_t* elem_bytes);

/* ---- boxes of one domain ----
 * A domain (one refinement level, the paper's MultiFab of boxes, §2) is a set
 * of boxes whose ghost zones on internal faces come from the neighbouring
 * box's interior instead of a boundary condition.  neighbors[6*b + f] is the
 * index of the box across face f (xlo, xhi, ylo, yhi, zlo, zhi) of box b, or
 * -1 to use the box's boundary condition on that face (periodic wrap of the
 * whole domain is expressed by linking the boxes at its two ends).  A
 * neighbour must have the same extents across the face, the same zone widths
 * and gamma; the descriptor's bc of a linked face is ignored.  The ghost fill
 * runs in x, then y, then z over all boxes, so edges and corners come from
 * the right boxes.  Synchronous; returns HYDRO_ERR_INVALID on a bad table.
 *
 * hydro_set_shared_dt(h, 1) makes every box advance with one dt per step, the
 * minimum over the boxes of their CFL steps (dt_dev == NULL in hydro_step),
 * as a level of one domain must.  A domain split into boxes then advances
 * exactly (bitwise) like the same domain in one box. */
int hydro_set_neighbors(hydro_handle* h, const int32_t* neighbors);
int hydro_set_shared_dt(hydro_handle* h, int enable);

/* ---- method variants ----
 * The paper says its hydro resembles Cholla's PPM scheme (§4) and prints no
 * formulas; the default method is PPM with the Colella & Woodward (1984)
 * limiter and an HLLC Riemann solver.  hydro_set_method selects, for every box
 * of the handle:
 *   limiter  HYDRO_LIMITER_CW84: van Leer slopes, 4th-order interfaces, CW84
 *            monotonicity limiter (default);
 *            HYDRO_LIMITER_CS08: Colella & Sekora (2008) extremum-preserving
 *            limiter (4th-order interfaces limited through second differences,
 *            smooth extrema kept unclipped, curvature bound C = 1.25);
 *   riemann  HYDRO_RIEMANN_HLLC (default), or HYDRO_RIEMANN_TWO_SHOCK: the
 *            two-shock approximation of Colella & Glaz (1985) (Newton on the
 *            Hugoniot velocity balance from the acoustic guess, Hugoniot star
 *            densities, linear interpolation across a rarefaction fan, Godunov
 *            flux of the state at x/t = 0).
 * Under HYDRO_LIMITER_CS08 the slope fields dq[3][5] of hydro_debug_fields
 * hold instead the interface value at the low face of each zone.  Applies to
 * the next step; HYDRO_ERR_INVALID on an unknown code. */
#define HYDRO_LIMITER_CW84 0
#define HYDRO_LIMITER_CS08 1
#define HYDRO_RIEMANN_HLLC 0
#define HYDRO_RIEMANN_TWO_SHOCK 1
int hydro_set_method(hydro_handle* h, int limiter, int riemann);

/* Launch configuration.  Every stage kernel covers all boxes of the handle in
 * one launch: the boxes' blocks are packed back to back through a work table
 * in the scratch head (block -> box and axis), so uneven boxes waste no
 * blocks.  hydro_step replays one step as a CUDA graph (captured on first use
 * for a given dt_dev, on a private stream) unless profiling is on or graphs
 * are switched off with hydro_use_graphs(h, 0).
 *
 * hydro_autotune times, for every stage kernel but the update and for each
 * compute type present, threads per block in {64, 128, 256} and two box
 * orders (as given, or largest work item first), `reps` launches each, keeps
 * the fastest and writes one record per tuned table (up to max_entries;
 * *nentries receives the count).  It does not change the state or the
 * simulated time (it refills ghosts and recomputes intermediates only), and
 * synchronises `stream` before returning. */
typedef struct hydro_tuning {
  char name[24];      /* fill_x, fill_y, fill_z, prim, flatten, slopes, trace, riemann, ctu1, ctu2, the line
                         tables, tile */
  int32_t precision;  /* HYDRO_FP64 or HYDRO_MIXED kernels */
  int32_t threads;    /* chosen threads per block (tile: 32 x (rows + 2)) */
  int32_t order;      /* 0: boxes in the given order, 1: largest work item first */
  float ms;           /* time of one launch with that choice */
  int32_t tile_rows;  /* tile: interior zone rows per tile (30 zones each); else 0 */
  int32_t tile_seg;   /* tile: z-planes per segment (0: the whole box); else 0 */
} hydro_tuning;
int hydro_autotune(hydro_handle* h, int reps, hydro_tuning* out, int max_entries, int* nentries, void* stream);
int hydro_use_graphs(hydro_handle* h, int enable);

/* Fused line stage.  For HYDRO_MIXED boxes under HYDRO_LIMITER_CW84 the slopes,
 * the limited parabolas, the characteristic tracing and the normal Riemann
 * solves of each axis run fused, one kernel for the x lines and one for the y
 * and z lines (tables "line_x" and "line_yz" in hydro_autotune): they depend
 * only on the zones of one line along the axis,
 * so the line's values stay in registers and only the traced edge states and
 * the normal fluxes reach HBM.  The arithmetic is that of the separate stages;
 * the slope fields dq of hydro_debug_fields are then not written for those
 * boxes, and the stage time of the fused kernel is reported under "trace".
 * Both transverse-correction stages of those boxes run zone by zone along
 * lines as well (tables "ctu1_line" and "ctu2_line"): the two edge states of
 * a zone share the flux differences across it, which are then read once.
 * On by default; hydro_fuse_lines(h, 0) runs the separate stages. */
int hydro_fuse_lines(hydro_handle* h, int enable);

/* Fused tile stage.  For HYDRO_MIXED boxes under HYDRO_LIMITER_CW84 one
 * kernel replaces the slope, tracing, Riemann, CTU and update stages: a block
 * advances a tile of 30 x rows interior zone columns of a box (with a one-zone
 * halo, 32 x (rows + 2) threads) over a segment of z-planes, marching in z
 * with the primitive state of each plane staged in shared memory and every
 * traced state and flux of the step kept on chip, then applies the FP64
 * update.  The results are bitwise those of the line stage (same arithmetic).
 * hydro_fuse_tiles(h, 1) switches it on (hydro_fuse_lines then applies to
 * nothing); hydro_autotune picks the tile rows (2 or 6) and the segment length
 * (16, 32, 64 planes or the whole box) and the box order by timing them;
 * hydro_set_tile_shape sets them directly (seg 0: the whole box).  Stage time
 * "tile" in hydro_profile_end.  Off by default. */
int hydro_fuse_tiles(hydro_handle* h, int enable);
int hydro_set_tile_shape(hydro_handle* h, int rows, int seg);

/* Persistent form.  hydro_persistent(h, 1) makes hydro_step advance every box
 * by all nsteps steps in one launch of one kernel: its blocks (as many as fit
 * on the GPU at once) take work blocks of the stage tables from a queue in
 * step, stage and box order, and a work block of a box's stage first waits
 * until the box's blocks of every earlier stage (of this and earlier steps)
 * are done.  Small or uneven boxes then flow through the stages without a
 * device-wide barrier between stages.  Every wait polls a bounded number of
 * times (hydro_set_spin_limit; about half a second by default): when one gives
 * up, the launch stops taking work and the next hydro_sync returns
 * HYDRO_ERR_TIMEOUT (the step it interrupted is incomplete).  The stage work
 * is the per-stage form's own code, so results are bitwise the same.  Needs
 * independent boxes (no hydro_set_neighbors links, no shared dt) and the fused
 * tile stage off; every stage table is rebuilt for 128-thread blocks, so
 * hydro_autotune is refused while the form is on.  Stage times are not
 * recorded by hydro_profile_* in this form.
 * hydro_set_spin_limit sets the polls before a wait gives up; stall_box >= 0
 * makes one wait of that box's second stage unreachable, which exercises the
 * give-up path (tests); -1 for normal operation. */
int hydro_persistent(hydro_handle* h, int enable);
int hydro_set_spin_limit(hydro_handle* h, int64_t polls, int stall_box);

/* Number of kernels this handle has launched since hydro_alloc (a ghost fill
 * is three kernels, every other stage one per compute type present), into
 * *count. */
int hydro_kernel_launches(hydro_handle* h, int64_t* count);

/* Per-stage device time.  Between hydro_profile_begin and hydro_profile_end
 * every stage launch is bracketed by a pair of CUDA events recorded on the
 * launching stream.  hydro_profile_end waits for those events and writes one
 * record per stage (up to max_stages, in launch order; *nstages receives the
 * number of stages): kernels launched and summed device milliseconds. */
typedef struct hydro_stage_time {
  char name[24];    /* fill_ghosts, prim, dt, flatten, slopes, trace, riemann, ctu1, ctu2, update */
  int64_t launches; /* kernels launched in the stage while profiling */
  double total_ms;  /* summed event time of those launches */
} hydro_stage_time;
int hydro_profile_begin(hydro_handle* h);
int hydro_profile_end(hydro_handle* h, hydro_stage_time* out, int max_stages, int* nstages);

/* Pipe-rate probes (diagnostics for rooflines): the measured FP64 and FP32
 * fused multiply-add rates of the current device, in flop/s (a multiply-add
 * counts 2), from two launches of kernels that do nothing but independent
 * multiply-add chains on every SM (about 0.3 s in all), and the device's SM
 * count.  Synchronous on `stream`. */
int hydro_measure_peaks(double* fp64_flops_per_s, double* fp32_flops_per_s, int32_t* sms, void* stream);

/* ---- time steps without any allocation by the caller ----
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need a time step: a process that
 * hands all device memory to its own pool at start-up and permits no further
 * allocation, or a latency-critical loop that cannot pay for cudaMalloc /
 * cudaFree (which may stall or synchronise the device).  hydro_compute_dt
 * needs a handle, and a handle needs a caller-allocated scratch buffer of
 * about 136 doubles per ghosted zone; this call needs neither.
 *
 * Writes dt_dev[b] = cfl / max over interior zones and axes a of
 * (|u_a| + c) / dx_a (the CFL step, cfl * min of dx_a / (|u_a| + c), up to
 * rounding) for boxes d[0..nboxes-1] whose states sit in state_dev with the
 * layout hydro_box_layout gives.  The speeds are formed by the same device
 * code as in hydro_compute_dt, so under the default limiter the two calls give
 * the same time steps bit for bit (under HYDRO_LIMITER_CS08 a handle forms its
 * primitive state with correctly rounded divides and the two agree to
 * rounding).  state_dev (input) and dt_dev (output, nboxes doubles) are
 * device pointers owned by the caller.  Its scratch is a fixed static device
 * array inside the library (about 100 KB, held by every GPU that loads the
 * library until the process exits) with room for HYDRO_NOALLOC_MAX_BOXES
 * boxes; a larger nboxes returns HYDRO_ERR_INVALID with a message saying so.
 * The call allocates nothing.
 *
 * The first call on a device looks up the device address of that array
 * (once per device, with the device current).  The call copies its box table
 * from host memory that lives only for the call, so it refuses to run while
 * `stream` is being captured into a CUDA graph (HYDRO_ERR_INVALID).  Every
 * call on a device shares the one array: each call rewrites the box table
 * and clears the per-box maxima before its kernels run, so calls ordered on
 * one stream are safe, but calls that may overlap on the GPU (different
 * streams, or several host threads) race and give wrong time steps.
 * Asynchronous on `stream`; the host buffers it reads are consumed before it
 * returns. */
#define HYDRO_NOALLOC_MAX_BOXES 1024
int hydro_compute_dt_noalloc(const hydro_box_desc* d, int nboxes, const double* state_dev, double* dt_dev,
                             void* stream);

/* ---- served form: continuous batching of independent requests ----
 * Source: data kept resident on the GPU and scratch served from a caching
 * pool (§3, memory management), and several independent boxes in flight at
 * once to keep the GPU busy (§4.A); each request is one box of §2.
 * A server owns one scheduler thread and a caller-owned device pool (the
 * memory budget).  hydro_submit copies a request (box, interior initial state,
 * step count) and returns at once with a ticket.  The scheduler admits queued
 * requests in submission order into up to max_active resident slots as slots
 * and pool memory free up (a later, smaller request may pass a head that does
 * not fit yet), uploads their states on a copy stream, and every tick advances
 * all resident requests by one step with one launch per stage over all of
 * them (each request keeps its own dt and precision).  Finished requests leave
 * the batch at once; their results are copied back while the next tick
 * computes.  A request's result does not depend on what else is resident: it
 * is bitwise the same alone and in the mix.  hydro_poll returns HYDRO_PENDING
 * until the result is on the host, then copies it out once.
 *
 * The pool holds the server's tables (a few hundred bytes per slot) and, per
 * resident request, its ghosted FP64 state and its scratch fields; a request
 * that could never fit the pool is refused with HYDRO_ERR_NOMEM at submit. */
typedef struct hydro_server hydro_server;
typedef struct hydro_server_config {
  void* pool_dev;      /* device pool, 256-byte aligned; may be NULL with dry_run */
  size_t pool_bytes;   /* budget: bytes of the pool */
  int32_t max_active;  /* resident slots, 1..4096 */
  int32_t dry_run;     /* 1: no GPU work (a tick completes one step of every resident
                          request instantly and the result equals the initial state);
                          for checks of the admission logic */
} hydro_server_config;
typedef struct hydro_request {
  hydro_box_desc desc;    /* the box, its boundary conditions and precision */
  const double* ic_host;  /* interior initial state [5][nz][ny][nx] (copied at submit) */
  int32_t nsteps;         /* steps to advance (>= 0), dt from the state each step */
} hydro_request;
typedef struct hydro_result {
  int32_t status;    /* HYDRO_OK, HYDRO_ERR_NONPHYSICAL, HYDRO_ERR_CUDA, ... */
  int32_t steps;     /* steps taken */
  double time;       /* simulated time reached */
  double queued_s;   /* wall seconds from submit to admission */
  double latency_s;  /* wall seconds from submit to the result on the host */
} hydro_result;
typedef struct hydro_server_stats {
  int64_t queued, active, admitted, finished, ticks, kernel_launches;
  int64_t bytes_in_use, peak_bytes, budget_bytes;
} hydro_server_stats;
int hydro_server_create(const hydro_server_config* cfg, hydro_server** out);
/* Stops admitting (queued requests are cancelled with HYDRO_ERR_INVALID),
 * finishes the resident ones, joins the scheduler and releases host state. */
int hydro_server_destroy(hydro_server* s);
/* Queues a request (its initial state is copied before the call returns) and
 * writes its ticket.  HYDRO_ERR_INVALID for a bad descriptor or step count,
 * HYDRO_ERR_NOMEM when the request could never fit the pool. */
int hydro_submit(hydro_server* s, const hydro_request* r, int64_t* ticket);
/* HYDRO_PENDING while running; HYDRO_OK once done (copies the interior result,
 * [5][nz][ny][nx] doubles, into out_host when it is not NULL; out_bytes must
 * match) and forgets the ticket; a failed request returns its error code. */
int hydro_poll(hydro_server* s, int64_t ticket, double* out_host, size_t out_bytes, hydro_result* info);
int hydro_server_get_stats(hydro_server* s, hydro_server_stats* out);

/* Thread-local description of the last error (never NULL). */
const char* hydro_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_GB300_H */
