// C ABI of the hydro library (declared in include/hydro.h): descriptor
// validation, the memory plan over caller-owned buffers, and the launch
// sequence of one step.  The library allocates no device memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hydro_internal.cuh"

using hydro::BoxRt;
using hydro::DevBox;
using hydro::HostBox;
using hydro::Plan;

struct hydro_handle {
  Plan plan;
  std::vector<HostBox> boxes;
  int device;
  size_t state_bytes, scratch_bytes;
  long long launches = 0;            // kernels launched through this handle
  bool profiling = false;            // record an event pair around every stage launch
  std::vector<cudaEvent_t> events;   // event pool (pairs), reused across sessions
  std::vector<int> rec_stage;        // stage of each recorded pair
  std::vector<int> rec_kernels;      // kernels launched inside each recorded pair
  std::vector<DevBox> dbox_host;     // host copy of the device box table
  // one step captured as a CUDA graph and replayed by hydro_step
  bool use_graphs = true;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const double* graph_dt = nullptr;  // dt_dev the graph was captured with
  int graph_kernels = 0;
};

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(HYDRO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr size_t ALIGN = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int validate(const hydro_box_desc& d, int i) {
  char buf[160];
  auto bad = [&](const char* what) {
    snprintf(buf, sizeof buf, "box %d: %s", i, what);
    return fail(HYDRO_ERR_INVALID, buf);
  };
  if (d.ng != HYDRO_NG) return bad("ng must be 4");
  if (d.nx < 4 || d.ny < 4 || d.nz < 4) return bad("every axis needs at least 4 interior zones");
  if ((long long)(d.nx + 2 * HYDRO_NG) * (d.ny + 2 * HYDRO_NG) * (d.nz + 2 * HYDRO_NG) > (1LL << 31))
    return bad("box too large (more than 2^31 zones with ghosts)");
  if (!(d.dx > 0.0) || !(d.dy > 0.0) || !(d.dz > 0.0)) return bad("zone widths must be > 0");
  if (!(d.gamma > 1.0)) return bad("gamma must be > 1");
  if (!(d.cfl > 0.0) || d.cfl > 1.0) return bad("cfl must be in (0, 1]");
  for (int a = 0; a < 3; a++) {
    const int lo = d.bc[2 * a], hi = d.bc[2 * a + 1];
    if (lo < HYDRO_BC_PERIODIC || lo > HYDRO_BC_REFLECT || hi < HYDRO_BC_PERIODIC || hi > HYDRO_BC_REFLECT)
      return bad("unknown boundary condition");
    if ((lo == HYDRO_BC_PERIODIC) != (hi == HYDRO_BC_PERIODIC)) return bad("periodic faces must pair");
  }
  if (d.precision != HYDRO_FP64 && d.precision != HYDRO_MIXED) return bad("precision must be HYDRO_FP64 or HYDRO_MIXED");
  return HYDRO_OK;
}

struct Geometry {
  std::vector<HostBox> boxes;
  size_t state_elems = 0;
  size_t table_bytes = 0, rt_bytes = 0, worktab_bytes = 0, persist_bytes = 0, head_bytes = 0;
  int cap[hydro::NTABLES][2] = {};  // work-table capacities (items)
  size_t work_bytes = 0, stage_elems = 0;
  size_t scratch_bytes = 0;
};

int plan_geometry(const hydro_box_desc* d, int nboxes, Geometry* g) {
  if (!d || nboxes <= 0) return fail(HYDRO_ERR_INVALID, "need at least one box descriptor");
  if (nboxes > 65535) return fail(HYDRO_ERR_INVALID, "at most 65535 boxes per handle");
  g->boxes.resize(nboxes);
  long long soff = 0, woff = 0, stoff = 0;
  for (int i = 0; i < nboxes; i++) {
    int rc = validate(d[i], i);
    if (rc) return rc;
    HostBox& hb = g->boxes[i];
    hb.d = d[i];
    hb.pitch = (long long)align_up((size_t)(d[i].nx + 2 * HYDRO_NG), 4);
    hb.plane = hb.pitch * (d[i].ny + 2 * HYDRO_NG);
    hb.vs = (long long)align_up((size_t)(hb.plane * (d[i].nz + 2 * HYDRO_NG)), 32);
    hb.interior = (long long)d[i].nx * d[i].ny * d[i].nz;
    hb.state_off = soff;
    hb.work_off = woff;
    hb.stage_off = stoff;
    soff += 5 * hb.vs;
    const size_t elem = d[i].precision == HYDRO_MIXED ? sizeof(float) : sizeof(double);
    woff += (long long)align_up((size_t)hydro::NFIELDS * hb.vs * elem, ALIGN);
    stoff += 5 * hb.interior;
  }
  g->state_elems = (size_t)soff;
  g->work_bytes = (size_t)woff;
  g->stage_elems = (size_t)stoff;
  g->table_bytes = align_up(sizeof(DevBox) * nboxes, ALIGN);
  g->rt_bytes = align_up(sizeof(BoxRt) * nboxes, ALIGN);
  int nmixed = 0;
  for (int i = 0; i < nboxes; i++) nmixed += d[i].precision == HYDRO_MIXED;
  size_t ints = 0;
  for (int t = 0; t < hydro::NTABLES; t++) {
    if (hydro::TABLE_PER_PRECISION[t]) {
      g->cap[t][0] = (nboxes - nmixed) * hydro::TABLE_ZDIM[t];
      g->cap[t][1] = nmixed * hydro::TABLE_ZDIM[t];
    } else {
      g->cap[t][0] = nboxes * hydro::TABLE_ZDIM[t];
      g->cap[t][1] = 0;
    }
    for (int s = 0; s < 2; s++)
      if (g->cap[t][s]) ints += 2 * (size_t)g->cap[t][s] + 1;
  }
  g->worktab_bytes = align_up(ints * sizeof(int), ALIGN);
  // persistent form: queue and error word, done counts, per-stage block
  // counts, and the work table of the per-box dt stage
  g->persist_bytes = align_up(sizeof(hydro::PersistHead), ALIGN) +
                     align_up(sizeof(unsigned long long) * nboxes, ALIGN) +
                     align_up(sizeof(long long) * (size_t)nboxes * (hydro::NPSTAGES + 1), ALIGN) +
                     align_up(sizeof(int) * (2 * (size_t)nboxes + 1), ALIGN);
  g->head_bytes = g->table_bytes + g->rt_bytes + g->worktab_bytes + g->persist_bytes;
  // the field area doubles as the staging buffer of hydro_upload/download
  g->scratch_bytes = g->head_bytes + std::max(g->work_bytes, g->stage_elems * sizeof(double));
  return HYDRO_OK;
}

int check_device(const hydro_handle* h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != h->device) return fail(HYDRO_ERR_INVALID, "handle used with a different current device");
  return HYDRO_OK;
}

int launched(cudaError_t e, const char* what) { return e == cudaSuccess ? HYDRO_OK : cuda_fail(e, what); }

void drop_graph(hydro_handle* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_dt = nullptr;
  h->graph_kernels = 0;
}

// Rebuilds one work table from its threads-per-block and order settings and
// copies it to the device (synchronously).
cudaError_t upload_table(hydro_handle* h, int t, int s) {
  hydro::WorkTable& w = h->plan.tab[t][s];
  if (w.capacity == 0) return cudaSuccess;
  std::vector<int> start(w.capacity + 1), item(w.capacity);
  w.nitems = hydro::build_table(h->plan, t, s, w.tpb, w.order, start.data(), item.data());
  w.blocks = start[w.nitems];
  cudaError_t e = cudaMemcpy(w.start, start.data(), sizeof(int) * (w.nitems + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(w.item, item.data(), sizeof(int) * w.nitems, cudaMemcpyHostToDevice);
  drop_graph(h);
  return e;
}

// Rebuilds the tables of the persistent form (defined with hydro_persistent).
cudaError_t setup_persistent(hydro_handle* h, bool on);

// Launches one stage, bracketed by timing events when profiling is on.
cudaError_t run_stage(hydro_handle* h, hydro::Stage st, cudaStream_t s, const double* dt_in = nullptr,
                      double* dt_out = nullptr, int advance = 0) {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (h->profiling) {
    const size_t need = 2 * (h->rec_stage.size() + 1);
    while (h->events.size() < need) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      h->events.push_back(e);
    }
    ev[0] = h->events[need - 2];
    ev[1] = h->events[need - 1];
    cudaError_t err = cudaEventRecord(ev[0], s);
    if (err != cudaSuccess) return err;
  }
  int n = 0;
  cudaError_t e = hydro::launch_stage(h->plan, st, s, dt_in, dt_out, advance, &n);
  if (e != cudaSuccess) return e;
  h->launches += n;
  if (h->profiling) {
    e = cudaEventRecord(ev[1], s);
    h->rec_stage.push_back((int)st);
    h->rec_kernels.push_back(n);
  }
  return e;
}

}  // namespace

namespace hydro {
void set_last_error(const std::string& msg) { g_err = msg; }

int box_layouts(const hydro_box_desc* d, int nboxes, hydro_layout* out) {
  if (!out) return fail(HYDRO_ERR_INVALID, "null output pointer");
  Geometry g;
  int rc = plan_geometry(d, nboxes, &g);
  if (rc) return rc;
  for (int i = 0; i < nboxes; i++) {
    const HostBox& hb = g.boxes[i];
    out[i].offset = hb.state_off;
    out[i].pitch = hb.pitch;
    out[i].plane = hb.plane;
    out[i].var_stride = hb.vs;
  }
  return HYDRO_OK;
}
}  // namespace hydro

namespace {

// The kernels of one step, in order, on stream s.
cudaError_t launch_step(hydro_handle* h, const double* dt_dev, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int st = hydro::ST_FILL; st < hydro::NSTAGES && e == cudaSuccess; st++) {
    if (st == hydro::ST_DT) e = run_stage(h, hydro::ST_DT, s, dt_dev, nullptr, 1);
    else e = run_stage(h, static_cast<hydro::Stage>(st), s);
  }
  return e;
}

// Captures one step (for this dt_dev) into a CUDA graph on a private stream.
int ensure_graph(hydro_handle* h, const double* dt_dev) {
  if (h->graph && h->graph_dt == dt_dev) return HYDRO_OK;
  drop_graph(h);
  cudaError_t e = cudaSuccess;
  if (!h->capture_stream) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "graph stream");
  const long long before = h->launches;
  e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  cudaError_t le = launch_step(h, dt_dev, h->capture_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->capture_stream, &graph);
  h->graph_kernels = (int)(h->launches - before);
  h->launches = before;
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return cuda_fail(e, "capturing the step graph");
  }
  h->graph_dt = dt_dev;
  return HYDRO_OK;
}

}  // namespace

namespace {

// Rebuilds every stage table for the persistent block size (or back to each
// table's default), the dt stage's table and the per-box block counts of
// each persistent stage.
cudaError_t setup_persistent(hydro_handle* h, bool on) {
  hydro::Plan& p = h->plan;
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < hydro::NTABLES && e == cudaSuccess; t++)
    for (int sl = 0; sl < 2 && e == cudaSuccess; sl++) {
      if (t == hydro::TB_TILE) continue;
      p.tab[t][sl].tpb = on ? hydro::PERSIST_THREADS : hydro::default_tpb(t);
      e = upload_table(h, t, sl);
    }
  if (e != cudaSuccess || !on) return e;
  const int n = p.nboxes;
  std::vector<long long> need((size_t)n * (hydro::NPSTAGES + 1), 0);
  for (int st = 0; st < hydro::NPSTAGES; st++) {
    int t, sl;
    hydro::persist_stage_table(st, &t, &sl);
    std::vector<long long> cnt(n, 0);
    if (t < 0) {
      for (int b = 0; b < n; b++) cnt[b] = h->boxes[b].active ? 1 : 0;
    } else if (hydro::persist_stage_runs(p, st)) {
      const hydro::WorkTable& w = p.tab[t][sl];
      std::vector<int> start(w.capacity + 1), item(w.capacity);
      const int ni = w.capacity ? hydro::build_table(p, t, sl, w.tpb, w.order, start.data(), item.data()) : 0;
      for (int i = 0; i < ni; i++) cnt[item[i] >> 3] += start[i + 1] - start[i];
    }
    for (int b = 0; b < n; b++) {
      long long* nb = need.data() + (size_t)b * (hydro::NPSTAGES + 1);
      if (st + 1 <= hydro::NPSTAGES) nb[st + 1] = nb[st] + cnt[b];
    }
  }
  // need[b][st]: blocks of box b in the stages before st; need[b][NPSTAGES]:
  // its blocks per step
  std::vector<int> dts(n + 1), dti(n);
  int k = 0;
  for (int b = 0; b < n; b++) {
    if (!h->boxes[b].active) continue;
    dts[k] = k;
    dti[k] = b * 8;
    k++;
  }
  dts[k] = k;
  p.p_dt_items = k;
  e = cudaMemcpy(p.p_need, need.data(), sizeof(long long) * need.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p.p_dt_start, dts.data(), sizeof(int) * (k + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && k) e = cudaMemcpy(p.p_dt_item, dti.data(), sizeof(int) * k, cudaMemcpyHostToDevice);
  int occ = 0, sms = 0;
  if (e == cudaSuccess) e = hydro::persist_occupancy(p, &occ);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  p.persist_grid = std::max(1, occ) * std::max(1, sms);
  return e;
}

}  // namespace

extern "C" {

const char* hydro_last_error(void) { return g_err.c_str(); }

int hydro_workspace_size(const hydro_box_desc* d, int nboxes, size_t* state_bytes, size_t* scratch_bytes) {
  if (!state_bytes || !scratch_bytes) return fail(HYDRO_ERR_INVALID, "null output pointer");
  Geometry g;
  int rc = plan_geometry(d, nboxes, &g);
  if (rc) return rc;
  *state_bytes = g.state_elems * sizeof(double);
  *scratch_bytes = g.scratch_bytes;
  return HYDRO_OK;
}

int hydro_box_layout(const hydro_box_desc* d, int nboxes, int box, hydro_layout* out) {
  if (!out) return fail(HYDRO_ERR_INVALID, "null output pointer");
  Geometry g;
  int rc = plan_geometry(d, nboxes, &g);
  if (rc) return rc;
  if (box < 0 || box >= nboxes) return fail(HYDRO_ERR_INVALID, "box index out of range");
  const HostBox& hb = g.boxes[box];
  out->offset = hb.state_off;
  out->pitch = hb.pitch;
  out->plane = hb.plane;
  out->var_stride = hb.vs;
  return HYDRO_OK;
}

int hydro_debug_fields(const hydro_box_desc* d, int nboxes, int box, int64_t* offset_bytes, int32_t* nfields,
                       int32_t* elem_bytes) {
  if (!offset_bytes || !nfields || !elem_bytes) return fail(HYDRO_ERR_INVALID, "null output pointer");
  Geometry g;
  int rc = plan_geometry(d, nboxes, &g);
  if (rc) return rc;
  if (box < 0 || box >= nboxes) return fail(HYDRO_ERR_INVALID, "box index out of range");
  *offset_bytes = (int64_t)g.head_bytes + g.boxes[box].work_off;
  *nfields = hydro::NFIELDS;
  *elem_bytes = d[box].precision == HYDRO_MIXED ? (int32_t)sizeof(float) : (int32_t)sizeof(double);
  return HYDRO_OK;
}

int hydro_alloc(const hydro_box_desc* d, int nboxes, void* state_dev, size_t state_bytes, void* scratch_dev,
                size_t scratch_bytes, hydro_handle** out) {
  if (!out) return fail(HYDRO_ERR_INVALID, "null output pointer");
  *out = nullptr;
  Geometry g;
  int rc = plan_geometry(d, nboxes, &g);
  if (rc) return rc;
  if (!state_dev || !scratch_dev) return fail(HYDRO_ERR_INVALID, "null device buffer");
  if ((reinterpret_cast<uintptr_t>(state_dev) | reinterpret_cast<uintptr_t>(scratch_dev)) % ALIGN)
    return fail(HYDRO_ERR_INVALID, "device buffers must be 256-byte aligned");
  if (state_bytes < g.state_elems * sizeof(double)) return fail(HYDRO_ERR_NOMEM, "state buffer too small");
  if (scratch_bytes < g.scratch_bytes) return fail(HYDRO_ERR_NOMEM, "scratch buffer too small");

  hydro_handle* h = new hydro_handle();
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice");
  }
  h->boxes = g.boxes;
  h->state_bytes = state_bytes;
  h->scratch_bytes = scratch_bytes;
  char* scratch = static_cast<char*>(scratch_dev);
  Plan& p = h->plan;
  p.nboxes = nboxes;
  p.boxes = h->boxes.data();
  p.dboxes = reinterpret_cast<DevBox*>(scratch);
  p.rt = reinterpret_cast<BoxRt*>(scratch + g.table_bytes);
  {
    int* ip = reinterpret_cast<int*>(scratch + g.table_bytes + g.rt_bytes);
    for (int t = 0; t < hydro::NTABLES; t++)
      for (int s = 0; s < 2; s++) {
        hydro::WorkTable& w = p.tab[t][s];
        w.capacity = g.cap[t][s];
        w.nitems = 0;
        w.blocks = 0;
        w.tpb = hydro::default_tpb(t);
        w.order = 0;
        w.start = w.item = nullptr;
        if (w.capacity) {
          w.start = ip;
          ip += w.capacity + 1;
          w.item = ip;
          ip += w.capacity;
        }
      }
  }
  {
    char* pp = scratch + g.table_bytes + g.rt_bytes + g.worktab_bytes;
    p.p_head = reinterpret_cast<hydro::PersistHead*>(pp);
    pp += align_up(sizeof(hydro::PersistHead), ALIGN);
    p.p_done = reinterpret_cast<unsigned long long*>(pp);
    pp += align_up(sizeof(unsigned long long) * nboxes, ALIGN);
    p.p_need = reinterpret_cast<long long*>(pp);
    pp += align_up(sizeof(long long) * (size_t)nboxes * (hydro::NPSTAGES + 1), ALIGN);
    p.p_dt_start = reinterpret_cast<int*>(pp);
    p.p_dt_item = p.p_dt_start + nboxes + 1;
  }
  p.state = static_cast<double*>(state_dev);
  p.work = reinterpret_cast<unsigned char*>(scratch + g.head_bytes);
  p.work_bytes = g.work_bytes;
  p.has_fp64 = false;
  p.has_mixed = false;
  p.max_interior = 0;
  p.max_ghosted = 0;
  for (int a = 0; a < 3; a++) p.max_n[a] = 0;

  std::vector<DevBox> table(nboxes);
  for (int i = 0; i < nboxes; i++) {
    const HostBox& hb = h->boxes[i];
    DevBox& db = table[i];
    memset(&db, 0, sizeof db);
    db.n[0] = hb.d.nx;
    db.n[1] = hb.d.ny;
    db.n[2] = hb.d.nz;
    db.precision = hb.d.precision;
    db.s[0] = 1;
    db.s[1] = hb.pitch;
    db.s[2] = hb.plane;
    db.vs = hb.vs;
    db.state_off = hb.state_off;
    db.work_off = hb.work_off;
    db.stage_off = hb.stage_off;
    const double dx[3] = {hb.d.dx, hb.d.dy, hb.d.dz};
    for (int a = 0; a < 3; a++) {
      db.dx[a] = dx[a];
      db.idx[a] = 1.0 / dx[a];
      p.max_n[a] = std::max(p.max_n[a], db.n[a]);
    }
    db.gamma = hb.d.gamma;
    db.igm1 = 1.0 / (hb.d.gamma - 1.0);
    db.gm1 = hb.d.gamma - 1.0;
    db.gamma_f = (float)db.gamma;
    db.igm1_f = (float)db.igm1;
    db.cfl = hb.d.cfl;
    for (int f = 0; f < 6; f++) db.bc[f] = hb.d.bc[f];
    p.max_interior = std::max(p.max_interior, hb.interior);
    if (hb.d.precision == HYDRO_MIXED) p.has_mixed = true;
    else p.has_fp64 = true;
    p.max_ghosted = std::max(p.max_ghosted, hb.vs);
  }
  h->dbox_host = table;
  e = cudaMemcpy(p.dboxes, table.data(), sizeof(DevBox) * nboxes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p.rt, 0, sizeof(BoxRt) * nboxes);
  if (e == cudaSuccess) e = cudaMemset(p.p_head, 0, sizeof(hydro::PersistHead));
  for (int t = 0; t < hydro::NTABLES && e == cudaSuccess; t++)
    for (int s = 0; s < 2 && e == cudaSuccess; s++) e = upload_table(h, t, s);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "hydro_alloc: writing the box table");
  }
  *out = h;
  return HYDRO_OK;
}

int hydro_free(hydro_handle* h) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  drop_graph(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  delete h;
  return HYDRO_OK;
}

int hydro_fill_ghosts(hydro_handle* h, void* stream) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  int rc = check_device(h);
  if (rc) return rc;
  return launched(run_stage(h, hydro::ST_FILL, static_cast<cudaStream_t>(stream)), "fill_ghosts launch");
}

int hydro_compute_dt(hydro_handle* h, double* dt_dev, void* stream) {
  if (!h || !dt_dev) return fail(HYDRO_ERR_INVALID, "null handle or dt pointer");
  int rc = check_device(h);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = run_stage(h, hydro::ST_PRIM, s);
  if (e == cudaSuccess) e = run_stage(h, hydro::ST_DT, s, nullptr, dt_dev, 0);
  return launched(e, "compute_dt launch");
}

int hydro_step(hydro_handle* h, const double* dt_dev, int nsteps, void* stream) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  if (nsteps < 0) return fail(HYDRO_ERR_INVALID, "nsteps must be >= 0");
  int rc = check_device(h);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nsteps == 0) return HYDRO_OK;
  if (h->plan.persistent) {
    // one launch for all nsteps steps; the queue and the done counts start at zero
    cudaError_t e = cudaMemsetAsync(&h->plan.p_head->queue, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->plan.p_done, 0, sizeof(unsigned long long) * h->plan.nboxes, s);
    if (e == cudaSuccess) e = hydro::launch_persistent(h->plan, dt_dev, nsteps, s);
    if (e != cudaSuccess) return cuda_fail(e, "persistent step launch");
    h->launches += 1;
    return HYDRO_OK;
  }
  if (h->use_graphs && !h->profiling) {
    rc = ensure_graph(h, dt_dev);
    if (rc) return rc;
    for (int i = 0; i < nsteps; i++) {
      cudaError_t e = cudaGraphLaunch(h->graph, s);
      if (e != cudaSuccess) return cuda_fail(e, "step graph launch");
      h->launches += h->graph_kernels;
    }
    return HYDRO_OK;
  }
  for (int i = 0; i < nsteps; i++) {
    cudaError_t e = launch_step(h, dt_dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
  }
  return HYDRO_OK;
}

int hydro_sync(hydro_handle* h, void* stream) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  int rc = check_device(h);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "hydro_sync");
  const int n = h->plan.nboxes;
  hydro::PersistHead ph;
  e = cudaMemcpy(&ph, h->plan.p_head, sizeof ph, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_sync: reading the persistent status");
  if (ph.err != 0) {
    // clear the error word and the signal-speed maxima the interrupted step
    // may have left, so that the next step starts clean
    e = cudaMemset(&h->plan.p_head->err, 0, sizeof(int));
    std::vector<BoxRt> rt0(n);
    if (e == cudaSuccess) e = cudaMemcpy(rt0.data(), h->plan.rt, sizeof(BoxRt) * n, cudaMemcpyDeviceToHost);
    for (BoxRt& r : rt0) r.smax = 0ull;
    if (e == cudaSuccess) e = cudaMemcpy(h->plan.rt, rt0.data(), sizeof(BoxRt) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "hydro_sync: clearing the persistent status");
    return fail(HYDRO_ERR_TIMEOUT,
                "persistent step: a block waited longer than the spin limit for the blocks of an earlier stage of "
                "its box and the launch gave up (the state of that step is incomplete)");
  }
  std::vector<BoxRt> rt(n);
  e = cudaMemcpy(rt.data(), h->plan.rt, sizeof(BoxRt) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_sync: reading status");
  int first = -1;
  for (int i = 0; i < n; i++) {
    if (rt[i].status && first < 0) first = i;
  }
  if (first < 0) return HYDRO_OK;
  for (int i = 0; i < n; i++) {
    if (rt[i].status) {
      e = cudaMemset(&h->plan.rt[i].status, 0, sizeof(unsigned));
      if (e != cudaSuccess) return cuda_fail(e, "hydro_sync: clearing status");
    }
  }
  char buf[160];
  snprintf(buf, sizeof buf, "box %d: nonphysical state (rho <= 0, p <= 0 or NaN) after step %u", first,
           rt[first].steps);
  return fail(HYDRO_ERR_NONPHYSICAL, buf);
}

int hydro_get_time(hydro_handle* h, double* time_host, void* stream) {
  if (!h || !time_host) return fail(HYDRO_ERR_INVALID, "null argument");
  int rc = check_device(h);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "hydro_get_time");
  const int n = h->plan.nboxes;
  std::vector<BoxRt> rt(n);
  e = cudaMemcpy(rt.data(), h->plan.rt, sizeof(BoxRt) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_get_time: reading times");
  for (int i = 0; i < n; i++) time_host[i] = rt[i].time;
  return HYDRO_OK;
}

int hydro_upload(hydro_handle* h, const double* state_host, size_t bytes, void* stream) {
  if (!h || !state_host) return fail(HYDRO_ERR_INVALID, "null argument");
  int rc = check_device(h);
  if (rc) return rc;
  size_t need = 0;
  for (const HostBox& hb : h->boxes) need += 5 * (size_t)hb.interior * sizeof(double);
  if (bytes != need) return fail(HYDRO_ERR_INVALID, "upload size does not match the boxes' interiors");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* stage = reinterpret_cast<double*>(h->plan.work);
  cudaError_t e = cudaMemcpyAsync(stage, state_host, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = hydro::launch_scatter(h->plan, stage, s);
  h->launches += 1;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return launched(e, "hydro_upload");
}

int hydro_download(hydro_handle* h, double* state_host, size_t bytes, void* stream) {
  if (!h || !state_host) return fail(HYDRO_ERR_INVALID, "null argument");
  int rc = check_device(h);
  if (rc) return rc;
  size_t need = 0;
  for (const HostBox& hb : h->boxes) need += 5 * (size_t)hb.interior * sizeof(double);
  if (bytes != need) return fail(HYDRO_ERR_INVALID, "download size does not match the boxes' interiors");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* stage = reinterpret_cast<double*>(h->plan.work);
  cudaError_t e = hydro::launch_gather(h->plan, stage, s);
  h->launches += 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(state_host, stage, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return launched(e, "hydro_download");
}

int hydro_set_neighbors(hydro_handle* h, const int32_t* neighbors) {
  if (!h || !neighbors) return fail(HYDRO_ERR_INVALID, "null argument");
  if (h->plan.persistent) return fail(HYDRO_ERR_INVALID, "hydro_set_neighbors: switch the persistent form off first");
  int rc = check_device(h);
  if (rc) return rc;
  const int n = h->plan.nboxes;
  std::vector<DevBox> t = h->dbox_host;
  for (int b = 0; b < n; b++)
    for (int f = 0; f < 6; f++) {
      const int o = neighbors[6 * b + f];
      char buf[160];
      if (o < -1 || o >= n) {
        snprintf(buf, sizeof buf, "box %d face %d: neighbour %d out of range", b, f, o);
        return fail(HYDRO_ERR_INVALID, buf);
      }
      t[b].nbr1[f] = o + 1;
      if (o < 0) continue;
      const int d = f / 2, e = (d + 1) % 3, g = (d + 2) % 3;
      const hydro_box_desc &A = h->boxes[b].d, &B = h->boxes[o].d;
      const int na[3] = {A.nx, A.ny, A.nz}, nb[3] = {B.nx, B.ny, B.nz};
      const double da[3] = {A.dx, A.dy, A.dz}, db[3] = {B.dx, B.dy, B.dz};
      if (na[e] != nb[e] || na[g] != nb[g] || nb[d] < HYDRO_NG) {
        snprintf(buf, sizeof buf, "box %d face %d: neighbour %d must match its extents across the face", b, f, o);
        return fail(HYDRO_ERR_INVALID, buf);
      }
      if (da[0] != db[0] || da[1] != db[1] || da[2] != db[2] || A.gamma != B.gamma) {
        snprintf(buf, sizeof buf, "box %d face %d: neighbour %d has other zone widths or gamma", b, f, o);
        return fail(HYDRO_ERR_INVALID, buf);
      }
    }
  cudaError_t e = cudaMemcpy(h->plan.dboxes, t.data(), sizeof(DevBox) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_set_neighbors");
  h->dbox_host = t;
  drop_graph(h);
  return HYDRO_OK;
}

int hydro_set_shared_dt(hydro_handle* h, int enable) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  if (enable && h->plan.persistent)
    return fail(HYDRO_ERR_INVALID, "hydro_set_shared_dt: switch the persistent form off first");
  h->plan.shared_dt = enable != 0;
  drop_graph(h);
  return HYDRO_OK;
}

int hydro_set_method(hydro_handle* h, int limiter, int riemann) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  if (limiter != HYDRO_LIMITER_CW84 && limiter != HYDRO_LIMITER_CS08)
    return fail(HYDRO_ERR_INVALID, "hydro_set_method: unknown limiter");
  if (riemann != HYDRO_RIEMANN_HLLC && riemann != HYDRO_RIEMANN_TWO_SHOCK)
    return fail(HYDRO_ERR_INVALID, "hydro_set_method: unknown Riemann solver");
  h->plan.limiter = limiter;
  h->plan.riemann = riemann;
  drop_graph(h);
  if (h->plan.persistent) return launched(setup_persistent(h, true), "hydro_set_method");
  return HYDRO_OK;
}

int hydro_fuse_lines(hydro_handle* h, int enable) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  h->plan.fuse_lines = enable != 0;
  drop_graph(h);
  if (h->plan.persistent) return launched(setup_persistent(h, true), "hydro_fuse_lines");
  return HYDRO_OK;
}


int hydro_persistent(hydro_handle* h, int enable) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  int rc = check_device(h);
  if (rc) return rc;
  hydro::Plan& p = h->plan;
  if (enable) {
    if (p.fuse_tiles) return fail(HYDRO_ERR_INVALID, "hydro_persistent: switch the fused tile stage off first");
    if (p.shared_dt) return fail(HYDRO_ERR_INVALID, "hydro_persistent: boxes with a shared dt are not independent");
    for (const DevBox& db : h->dbox_host)
      for (int f = 0; f < 6; f++)
        if (db.nbr1[f]) return fail(HYDRO_ERR_INVALID, "hydro_persistent: linked boxes are not independent");
  }
  p.persistent = enable != 0;
  return launched(setup_persistent(h, p.persistent), "hydro_persistent");
}

int hydro_set_spin_limit(hydro_handle* h, int64_t polls, int stall_box) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  if (polls < 0) return fail(HYDRO_ERR_INVALID, "hydro_set_spin_limit: polls must be >= 0");
  if (stall_box < -1 || stall_box >= h->plan.nboxes) return fail(HYDRO_ERR_INVALID, "hydro_set_spin_limit: bad box");
  h->plan.spin_limit = polls;
  h->plan.stall_box = stall_box;
  return HYDRO_OK;
}

int hydro_fuse_tiles(hydro_handle* h, int enable) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  int rc = check_device(h);
  if (rc) return rc;
  if (enable) {
    if (h->plan.persistent) return fail(HYDRO_ERR_INVALID, "hydro_fuse_tiles: switch the persistent form off first");
    cudaError_t e = hydro::prepare_tile_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "hydro_fuse_tiles");
  }
  h->plan.fuse_tiles = enable != 0;
  return launched(upload_table(h, hydro::TB_TILE, 1), "hydro_fuse_tiles");
}

int hydro_set_tile_shape(hydro_handle* h, int rows, int seg) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  if (rows != hydro::TILE_TYS[0] && rows != hydro::TILE_TYS[1])
    return fail(HYDRO_ERR_INVALID, "hydro_set_tile_shape: rows must be 2 or 6");
  if (seg < 0) return fail(HYDRO_ERR_INVALID, "hydro_set_tile_shape: seg must be >= 0");
  int rc = check_device(h);
  if (rc) return rc;
  h->plan.tile_ty = rows;
  h->plan.tile_seg = seg;
  return launched(upload_table(h, hydro::TB_TILE, 1), "hydro_set_tile_shape");
}

int hydro_use_graphs(hydro_handle* h, int enable) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  h->use_graphs = enable != 0;
  if (!h->use_graphs) drop_graph(h);
  return HYDRO_OK;
}

namespace {

// The state of every FP32 box copied into (or back from) its scratch fields
// that the fused tile stage leaves unused (from the traced-state fields on).
cudaError_t save_mixed_state(hydro_handle* h, bool restore, cudaStream_t s) {
  const hydro::Plan& p = h->plan;
  for (int b = 0; b < p.nboxes; b++) {
    const HostBox& hb = h->boxes[b];
    if (hb.d.precision != HYDRO_MIXED) continue;
    double* st = p.state + hb.state_off;
    unsigned char* bk = p.work + hb.work_off + (size_t)hydro::FLD_QM * hb.vs * sizeof(float);
    const size_t bytes = 5 * (size_t)hb.vs * sizeof(double);
    cudaError_t e = restore ? cudaMemcpyAsync(st, bk, bytes, cudaMemcpyDeviceToDevice, s)
                            : cudaMemcpyAsync(bk, st, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Tile rows, z-segment length and box order of the fused tile stage: every
// combination timed over `reps` launches (each launch updates the state, which
// is saved before and restored after), the fastest kept.
cudaError_t tune_tiles(hydro_handle* h, int reps, cudaStream_t s, cudaEvent_t* ev, hydro_tuning* out, int max_entries,
                       int* n) {
  hydro::Plan& p = h->plan;
  hydro::WorkTable& w = p.tab[hydro::TB_TILE][1];
  const int segs[4] = {16, 32, 64, 0};
  int best_ty = p.tile_ty, best_seg = p.tile_seg, best_order = w.order;
  float best_ms = 0.f;
  bool first = true;
  // the repeated updates may flag states nonphysical: the runtime records
  // (status flags) are saved and restored too
  std::vector<BoxRt> rt_saved(p.nboxes);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(rt_saved.data(), p.rt, sizeof(BoxRt) * p.nboxes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = save_mixed_state(h, false, s);
  for (int ti = 0; ti < 2 && e == cudaSuccess; ti++)
    for (int si = 0; si < 4 && e == cudaSuccess; si++)
      for (int o = 0; o < 2 && e == cudaSuccess; o++) {
        p.tile_ty = hydro::TILE_TYS[ti];
        p.tile_seg = segs[si];
        w.order = o;
        e = upload_table(h, hydro::TB_TILE, 1);
        if (e == cudaSuccess) e = hydro::launch_table(p, hydro::TB_TILE, 1, s);  // warm
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        for (int r = 0; r < reps && e == cudaSuccess; r++) e = hydro::launch_table(p, hydro::TB_TILE, 1, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        ms /= reps;
        if (e == cudaSuccess && (first || ms < best_ms)) {
          best_ms = ms;
          best_ty = p.tile_ty;
          best_seg = p.tile_seg;
          best_order = o;
          first = false;
        }
      }
  if (e == cudaSuccess) e = save_mixed_state(h, true, s);
  p.tile_ty = best_ty;
  p.tile_seg = best_seg;
  w.order = best_order;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(p.rt, rt_saved.data(), sizeof(BoxRt) * p.nboxes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = upload_table(h, hydro::TB_TILE, 1);
  if (e == cudaSuccess && *n < max_entries) {
    memset(&out[*n], 0, sizeof out[*n]);
    snprintf(out[*n].name, sizeof out[*n].name, "%s", hydro::TABLE_NAMES[hydro::TB_TILE]);
    out[*n].precision = HYDRO_MIXED;
    out[*n].threads = 32 * (best_ty + 2);
    out[*n].order = best_order;
    out[*n].ms = best_ms;
    out[*n].tile_rows = best_ty;
    out[*n].tile_seg = best_seg;
  }
  (*n)++;
  return e;
}

}  // namespace

int hydro_autotune(hydro_handle* h, int reps, hydro_tuning* out, int max_entries, int* nentries, void* stream) {
  if (!h || !nentries || (max_entries > 0 && !out)) return fail(HYDRO_ERR_INVALID, "null argument");
  if (reps < 1) return fail(HYDRO_ERR_INVALID, "reps must be >= 1");
  int rc = check_device(h);
  if (rc) return rc;
  if (h->plan.persistent)
    return fail(HYDRO_ERR_INVALID, "hydro_autotune: the persistent form fixes the block size; tune before switching "
                                   "it on");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  hydro::Plan& p = h->plan;
  // scratch in a consistent state for the current interior, time not advanced
  cudaError_t e = run_stage(h, hydro::ST_FILL, s);
  if (e == cudaSuccess) e = run_stage(h, hydro::ST_PRIM, s);
  if (e == cudaSuccess) e = run_stage(h, hydro::ST_DT, s, nullptr, nullptr, 0);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_autotune: first pass");
  cudaEvent_t ev[2];
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_autotune: events");
  const int tpbs[3] = {64, 128, 256};
  int n = 0;
  // pipeline order, so that every table is tuned on valid inputs
  const int order[] = {hydro::TB_FILL_X,  hydro::TB_FILL_Y,  hydro::TB_FILL_Z, hydro::TB_PRIM,
                       hydro::TB_FLATTEN, hydro::TB_SLOPES,  hydro::TB_TRACE,  hydro::TB_RIEMANN,
                       hydro::TB_LINE_X,  hydro::TB_LINE_YZ, hydro::TB_CTU1,   hydro::TB_CTU1_LINE,
                       hydro::TB_CTU2,    hydro::TB_CTU2_LINE, hydro::TB_TILE};
  for (int t : order) {
    for (int sl = 0; sl < 2; sl++) {
      hydro::WorkTable& w = p.tab[t][sl];
      if (w.capacity == 0) continue;
      // tune what the step runs: the line table, or the three stages it replaces
      const bool fused = hydro::line_fused(p, sl);
      const bool line = t == hydro::TB_LINE_X || t == hydro::TB_LINE_YZ || t == hydro::TB_CTU1_LINE ||
                        t == hydro::TB_CTU2_LINE;
      const bool replaced = t == hydro::TB_SLOPES || t == hydro::TB_TRACE || t == hydro::TB_RIEMANN ||
                            t == hydro::TB_CTU1 || t == hydro::TB_CTU2;
      if (t == hydro::TB_TILE) {
        if (!hydro::tile_fused(p, sl)) continue;
        e = tune_tiles(h, reps, s, ev, out, max_entries, &n);
        if (e != cudaSuccess) break;
        continue;
      }
      if (hydro::tile_fused(p, sl) && (line || replaced)) continue;
      if (line ? !fused : fused && replaced) continue;
      int best_tpb = w.tpb, best_order = w.order;
      float best_ms = 0.f;
      bool first = true;
      for (int ti = 0; ti < 3 && e == cudaSuccess; ti++)
        for (int o = 0; o < 2 && e == cudaSuccess; o++) {
          w.tpb = tpbs[ti];
          w.order = o;
          e = upload_table(h, t, sl);
          if (e == cudaSuccess) e = hydro::launch_table(p, t, sl, s);  // warm
          if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
          for (int r = 0; r < reps && e == cudaSuccess; r++) e = hydro::launch_table(p, t, sl, s);
          if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
          if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
          ms /= reps;
          if (e == cudaSuccess && (first || ms < best_ms)) {
            best_ms = ms;
            best_tpb = w.tpb;
            best_order = w.order;
            first = false;
          }
        }
      if (e != cudaSuccess) break;
      w.tpb = best_tpb;
      w.order = best_order;
      e = upload_table(h, t, sl);
      if (e == cudaSuccess) e = hydro::launch_table(p, t, sl, s);  // valid outputs for the next table
      if (n < max_entries) {
        memset(&out[n], 0, sizeof out[n]);
        snprintf(out[n].name, sizeof out[n].name, "%s", hydro::TABLE_NAMES[t]);
        out[n].precision = hydro::TABLE_PER_PRECISION[t] && sl == 1 ? HYDRO_MIXED : HYDRO_FP64;
        out[n].threads = best_tpb;
        out[n].order = best_order;
        out[n].ms = best_ms;
      }
      n++;
    }
    if (e != cudaSuccess) break;
  }
  // the tuning launches of k_prim left their maxima behind: reset them
  if (e == cudaSuccess) e = run_stage(h, hydro::ST_DT, s, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "hydro_autotune");
  *nentries = n;
  return HYDRO_OK;
}

int hydro_kernel_launches(hydro_handle* h, int64_t* count) {
  if (!h || !count) return fail(HYDRO_ERR_INVALID, "null argument");
  *count = h->launches;
  return HYDRO_OK;
}

int hydro_profile_begin(hydro_handle* h) {
  if (!h) return fail(HYDRO_ERR_INVALID, "null handle");
  h->rec_stage.clear();
  h->rec_kernels.clear();
  h->profiling = true;
  return HYDRO_OK;
}

int hydro_profile_end(hydro_handle* h, hydro_stage_time* out, int max_stages, int* nstages) {
  if (!h || !nstages || (max_stages > 0 && !out)) return fail(HYDRO_ERR_INVALID, "null argument");
  h->profiling = false;
  double ms[hydro::NSTAGES] = {0};
  long long n[hydro::NSTAGES] = {0};
  for (size_t r = 0; r < h->rec_stage.size(); r++) {
    cudaError_t e = cudaEventSynchronize(h->events[2 * r + 1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, h->events[2 * r], h->events[2 * r + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "hydro_profile_end");
    ms[h->rec_stage[r]] += t;
    n[h->rec_stage[r]] += h->rec_kernels[r];
  }
  h->rec_stage.clear();
  h->rec_kernels.clear();
  *nstages = hydro::NSTAGES;
  for (int s = 0; s < hydro::NSTAGES && s < max_stages; s++) {
    memset(&out[s], 0, sizeof out[s]);
    snprintf(out[s].name, sizeof out[s].name, "%s", hydro::STAGE_NAMES[s]);
    out[s].launches = n[s];
    out[s].total_ms = ms[s];
  }
  return HYDRO_OK;
}

}  // extern "C"
