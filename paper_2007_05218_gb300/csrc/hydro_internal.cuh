// Internal declarations shared by the CUDA translation units of the hydro
// library (box table, per-box runtime record, scratch field map, launchers).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/hydro.h"

namespace hydro {

constexpr int NG = HYDRO_NG;

// Method parameters (floors and CW84 flattening constants).
constexpr double SMALL_DENS = 1e-12;
constexpr double SMALL_PRES = 1e-12;
constexpr double FLAT_EPS = 0.33;
constexpr double FLAT_OMEGA1 = 0.75;
constexpr double FLAT_OMEGA2 = 10.0;

// Scratch fields of one box, each a full ghosted-box grid of doubles with the
// state's pitch/plane strides:
//   q[5] primitive (rho,u,v,w,p), c sound speed, chi flattening,
//   qm[d][5] / qp[d][5] traced left-/right-edge states in the normal frame of d
//   (rho, u_n, u_t1, u_t2, p with t1 = (d+1)%3, t2 = (d+2)%3),
//   f0[d][5] normal fluxes, f1[pair][5] singly corrected fluxes for the ordered
//   pairs (d,e) = xy,xz,yx,yz,zx,zy, f[d][5] final fluxes (conserved x,y,z order),
//   dq[d][5] limited slopes of the normal-frame variables of axis d,
//   um[d][4] / up[d][4] conserved momenta (normal frame) and total energy of
//   the left-/right-edge states,
//   ic = 1/c and cr = c/rho of each zone (FP64 boxes; for the tracing).
// Flux of a d-face between zones Z-s_d and Z is stored at zone Z.
enum Field : int {
  FLD_Q = 0,
  FLD_C = 5,
  FLD_CHI = 6,
  FLD_QM = 7,
  FLD_QP = 22,
  FLD_F0 = 37,
  FLD_F1 = 52,
  FLD_F = 82,
  FLD_DQ = 97,
  FLD_UM = 112,
  FLD_UP = 124,
  FLD_IC = 136,
  FLD_CR = 137,
  NFIELDS = 138
};

// Per-box geometry as the kernels see it (lives in the head of scratch).
struct DevBox {
  int n[3];
  int precision;
  long long s[3];         // element strides of i, j, k
  long long vs;           // element stride between fields/variables
  long long state_off;    // first state element of this box
  long long work_off;     // byte offset of this box's fields in the field area
  long long stage_off;    // first element of this box in the compact host staging layout
  double dx[3];
  double idx[3];          // 1/dx
  double gamma;
  double igm1;            // 1/(gamma-1)
  double gm1;             // gamma-1
  double cfl;
  int bc[6];
  float gamma_f, igm1_f;  // FP32 copies for the mixed-precision kernels
  int nbr1[6];            // per face: 1 + index of the box whose interior fills its ghosts, 0: use bc
  int pad2[2];
};

// Per-box runtime record (lives in scratch, after the box table).
struct BoxRt {
  unsigned long long smax;  // max over interior zones/axes of (|u|+c)/dx, as non-negative double bits
  double dt;                // time step of the current update
  double time;              // simulated time advanced so far
  unsigned int status;      // device error flags (STATUS_*)
  unsigned int steps;       // updates applied
  float dtdx_f[3];          // FP32 dt/dx per axis for the mixed-precision kernels
  float pad;
  // FP64 dt/dx per axis and the transverse-correction factors dt/(3 dx) and
  // dt/(2 dx), each formed once per step by the time-step kernel (as the
  // products (dt * (1/dx)) * (1/3) and 0.5 * (dt * (1/dx))) instead of in
  // every thread of the FP64 stages
  double dtdx[3], dtdx3[3], dtdx2[3];
};

constexpr unsigned STATUS_NONPHYSICAL = 1u;

// Geometry computed on the host for one box.
struct HostBox {
  hydro_box_desc d;
  long long pitch, plane, vs;
  long long state_off, work_off, stage_off;  // work_off in bytes
  long long interior;  // nx*ny*nz
  bool active = true;  // false: a free slot of a server plan (no work items)
};

// Work tables: every launch of a stage covers a list of work items (one box,
// or one box and axis / axis pair) whose blocks are packed back to back, so
// boxes of uneven size waste no blocks.  Block b of a launch belongs to the
// item i with start[i] <= b < start[i+1]; item[i] = box * 8 + axis (or pair).
enum TableId : int {
  TB_FILL_X = 0,
  TB_FILL_Y,
  TB_FILL_Z,
  TB_PRIM,
  TB_UPDATE,
  TB_FLATTEN,
  TB_SLOPES,
  TB_TRACE,
  TB_RIEMANN,
  TB_CTU1,
  TB_CTU2,
  TB_LINE_X,   // fused slopes + tracing + normal Riemann solves along x (FP32 boxes)
  TB_LINE_YZ,  // the same along y (item z = 0) and z (item z = 1)
  TB_CTU2_LINE,  // CTU stage 2 by zones along lines (FP32 boxes)
  TB_CTU1_LINE,  // CTU stage 1 by zones along lines (FP32 boxes)
  TB_TILE,       // fused tile stage: tracing, CTU, solves and update per z-marching tile (FP32 boxes)
  NTABLES
};
constexpr int TABLE_ZDIM[NTABLES] = {1, 1, 1, 1, 1, 1, 3, 3, 3, 6, 3, 1, 2, 3, 6, 1};
// tables of the precision-specific stage kernels exist once per compute type
constexpr bool TABLE_PER_PRECISION[NTABLES] = {false, false, false, false, false, true, true, true, true, true, true,
                                               true, true, true, true, true};
// tile shapes of the fused tile stage: 30 x TILE_TY[k] interior zone columns
// per block (32 x (TY + 2) threads), marching over z-segments of a chosen length
constexpr int TILE_TYS[2] = {2, 6};
// the fused line stage runs for FP32 boxes only (slot 1): the FP64 stages are
// bound by the FP64 pipe, which fusion does not relieve
constexpr bool LINE_FUSED_SLOT[2] = {false, true};
// zones a warp produces along x in the fused line stage (lanes 3..29 of 32;
// the other lanes supply the stencil's neighbours by shuffle) and traced zones
// a thread produces along y or z (walking a column)
constexpr int LINE_X_OUT = 27;
constexpr int LINE_SEG = 16;

struct WorkTable {
  int* start;      // device, nitems + 1 entries (start[nitems] = blocks)
  int* item;       // device, nitems entries
  int nitems;      // 0: nothing to launch
  int capacity;    // items the device arrays hold
  int blocks;      // blocks of one launch
  int tpb;         // threads per block
  int order;       // 0: box order, 1: largest items first
};

// Persistent form: one kernel advances every box of a handle by K steps,
// its blocks taking work blocks of the stage tables from a queue in step and
// stage order; a block of a stage waits (bounded) until the box's blocks of
// every earlier stage are done.  The stages, in the order of a step:
enum PStage : int {
  PS_FILL_X = 0, PS_FILL_Y, PS_FILL_Z, PS_PRIM, PS_DT,
  PS_FLATTEN_D, PS_FLATTEN_F, PS_SLOPES_D, PS_SLOPES_F, PS_TRACE_D, PS_TRACE_F, PS_LINE_X, PS_LINE_YZ,
  PS_RIEMANN_D, PS_RIEMANN_F, PS_CTU1_D, PS_CTU1_F, PS_CTU1_LINE, PS_CTU2_D, PS_CTU2_F, PS_CTU2_LINE,
  PS_UPDATE, NPSTAGES
};
constexpr int PERSIST_THREADS = 128;  // every stage table is built for this block size in that form
constexpr int PERSIST_CHUNK = 8;      // work blocks a block takes per queue access
constexpr long long DEFAULT_SPIN_LIMIT = 1LL << 22;  // polls (about 128 ns apart) before a wait gives up

// Queue and error word of the persistent form (device, scratch head), then
// done[nboxes] (unsigned long long: blocks of the box finished) and
// need[nboxes][NPSTAGES + 1] (blocks of the box before each stage within a
// step; the last entry is the box's blocks per step).
struct PersistHead {
  unsigned long long queue;
  int err;
  int pad;
};

// Host-side plan of a handle.
struct Plan {
  int nboxes;
  HostBox* boxes;      // host array [nboxes]
  DevBox* dboxes;      // device table (in scratch)
  BoxRt* rt;           // device runtime records (in scratch)
  double* state;
  unsigned char* work; // start of the per-box field area (in scratch)
  size_t work_bytes;   // bytes of the field area
  bool has_fp64, has_mixed;
  int max_n[3];        // max interior extent per axis over boxes
  long long max_ghosted, max_interior;
  WorkTable tab[NTABLES][2];  // [table][0: FP64 boxes (or all boxes), 1: mixed boxes]
  bool shared_dt = false;     // one dt for all boxes: the minimum of their CFL steps
  int limiter = HYDRO_LIMITER_CW84;   // reconstruction variant of every box
  int riemann = HYDRO_RIEMANN_HLLC;   // Riemann solver of every box
  bool fuse_lines = true;             // fused line stage for FP32 boxes (CW84 limiter)
  bool fuse_tiles = false;            // fused tile stage for FP32 boxes (CW84 limiter)
  int tile_ty = 6;                    // tile rows (one of TILE_TYS)
  int tile_seg = 64;                  // z-planes per tile segment (0: the whole box)
  // persistent form (hydro_persistent)
  bool persistent = false;
  PersistHead* p_head = nullptr;      // device
  unsigned long long* p_done = nullptr;  // device [nboxes]
  long long* p_need = nullptr;        // device [nboxes][NPSTAGES + 1]
  int* p_dt_start = nullptr;          // device: work table of the per-box dt stage
  int* p_dt_item = nullptr;
  int p_dt_items = 0;
  long long spin_limit = DEFAULT_SPIN_LIMIT;
  int stall_box = -1;                 // test hook: a wait of this box that can never be met
  int persist_grid = 0;               // blocks of the persistent launch
};

// Whether precision slot `slot` runs the fused tile stage under this plan
// (it replaces the slope, tracing, Riemann, CTU and update stages there).
inline bool tile_fused(const Plan& p, int slot) {
  return LINE_FUSED_SLOT[slot] && p.fuse_tiles && p.limiter == HYDRO_LIMITER_CW84;
}

// Whether precision slot `slot` runs the fused line stage under this plan.
inline bool line_fused(const Plan& p, int slot) {
  return LINE_FUSED_SLOT[slot] && p.fuse_lines && p.limiter == HYDRO_LIMITER_CW84 && !tile_fused(p, slot);
}

// Blocks of the fused tile stage for one box: tiles of 30 x ty columns times
// z-segments of seg planes (seg <= 0: one segment).
inline long long tile_blocks(const hydro_box_desc& d, int ty, int seg) {
  const long long ntx = (d.nx + 29) / 30, nty = (d.ny + ty - 1) / ty;
  const int sl = seg > 0 ? seg : d.nz;
  return ntx * nty * ((d.nz + sl - 1) / sl);
}

// Threads per block each table starts with (before any autotuning).
int default_tpb(int table);
// Cells (threads) of work item (box, z) of a table.
long long item_volume(const hydro_box_desc& d, int table, int z);
// Fills the host copies of a table for the given precision slot, threads per
// block and order; returns the number of items.
int build_table(const Plan& p, int table, int slot, int tpb, int order, int* start, int* item);

// Stages of one step, in launch order.  Each stage is one kernel, except the
// ghost fill (three kernels: x, y, z).
enum Stage : int {
  ST_FILL = 0,
  ST_PRIM,
  ST_DT,
  ST_FLATTEN,
  ST_SLOPES,
  ST_TRACE,
  ST_RIEMANN,
  ST_CTU1,
  ST_CTU2,
  ST_TILE,
  ST_UPDATE,
  NSTAGES
};
extern const char* const STAGE_NAMES[NSTAGES];

// Launches one stage for every box of the plan (hydro_kernels.cu),
// asynchronously on `stream`; *launched receives the number of kernels.
// ST_DT uses dt_in[b] when dt_in is not null (else cfl/smax), writes dt_out[b]
// when dt_out is not null, and advances the per-box time when `advance` is set.
cudaError_t launch_stage(const Plan& p, Stage st, cudaStream_t stream, const double* dt_in, double* dt_out,
                         int advance, int* launched);
// Launches the kernel of one work table for one precision slot (every table
// but TB_UPDATE; used by the autotuner, which must not change the state).
cudaError_t launch_table(const Plan& p, int table, int slot, cudaStream_t stream);
extern const char* const TABLE_NAMES[NTABLES];
cudaError_t launch_scatter(const Plan& p, const double* stage, cudaStream_t stream);
// Sets the thread-local message returned by hydro_last_error (hydro_api.cu).
void set_last_error(const std::string& msg);
// Validates d[0..nboxes-1] and writes every box's place in the state buffer
// (what hydro_box_layout gives for each box) in one pass (hydro_api.cu).
int box_layouts(const hydro_box_desc* d, int nboxes, hydro_layout* out);
cudaError_t launch_gather(const Plan& p, double* stage, cudaStream_t stream);
// Allows the fused tile kernels their dynamic shared memory (once per
// process; call outside stream capture).
cudaError_t prepare_tile_kernels();
// The table and precision slot behind each persistent stage, and whether the
// plan runs that stage (its table then holds the stage's blocks).
void persist_stage_table(int st, int* table, int* slot);
bool persist_stage_runs(const Plan& p, int st);
// Blocks per SM of the persistent kernel for this plan's method.
cudaError_t persist_occupancy(const Plan& p, int* blocks_per_sm);
// One launch of the persistent kernel: nsteps steps of every box, dt from
// dt_in or from the state.  The caller has zeroed the queue and done counts.
cudaError_t launch_persistent(const Plan& p, const double* dt_in, int nsteps, cudaStream_t stream);

}  // namespace hydro
