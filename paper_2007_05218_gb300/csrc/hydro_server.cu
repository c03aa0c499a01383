// Served form: independent hydro requests solved with continuous batching.
//
// The paper keeps simulation data resident on the GPU and serves its frequent
// scratch allocations from a caching pool (§3, memory management); it runs
// several CUDA streams over small boxes to keep the GPU busy (§4.A).  The
// server does both for a stream of independent requests: every request's
// state and scratch live in one caller-owned device pool (the memory budget),
// requests are admitted into fixed slots as slots and memory free up, and
// each tick advances every resident request by one step through the same
// batched launches (one launch per stage over all resident boxes, each box
// with its own dt).  Uploads of newly admitted requests run on a copy stream
// and results of finished requests are copied back while the next tick
// computes.  A request's arithmetic does not depend on its neighbours in the
// batch, so its result is bitwise the same alone and in the mix.
//
// One scheduler thread owns all CUDA work of a server; hydro_submit and
// hydro_poll only touch host state under a mutex.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hydro_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t ALIGN = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail(int code, const std::string& msg) {
  hydro::set_last_error(msg);
  return code;
}

// First-fit allocator over [0, size) with 256-byte granularity and coalescing.
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes, ALIGN);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes, ALIGN);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

enum ReqState { RS_QUEUED, RS_ACTIVE, RS_FINISHING, RS_DONE };

struct Request {
  int64_t ticket;
  hydro_box_desc d;
  int nsteps;
  std::vector<double> ic;      // host copy of the interior initial state
  std::vector<double> result;  // interior result, [5][nz][ny][nx]
  hydro::HostBox hb;           // geometry; offsets into the pool once admitted
  size_t state_off = 0, state_bytes = 0, work_off = 0, work_bytes = 0;
  int slot = -1;
  int steps_done = 0;
  ReqState st = RS_QUEUED;
  int status = HYDRO_OK;
  int steps = 0;
  double time = 0.0;
  Clock::time_point t_submit, t_admit, t_done;
  cudaEvent_t ev = nullptr;  // upload done (active) / last step done (finishing)
};

}  // namespace

struct hydro_server {
  hydro_server_config cfg{};
  bool dry = false;
  int device = 0;
  unsigned char* pool = nullptr;  // device
  size_t head_bytes = 0;
  Pool mem;  // the part of the pool after the head
  hydro::Plan plan{};
  std::vector<hydro::HostBox> slots;
  std::vector<Request*> slot_req;
  std::vector<hydro::DevBox> dbox_host;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<Request*> queue;
  std::vector<Request*> finishing;
  int64_t next_ticket = 1;
  long long ticks = 0, admitted = 0, finished = 0, launches = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  cudaStream_t compute = nullptr, copy = nullptr;
  std::string worker_error;
  // pinned staging of the per-tick box table and work tables (double buffered)
  unsigned char* staging[2] = {nullptr, nullptr};
  cudaEvent_t staging_ev[2] = {nullptr, nullptr};
  int staging_next = 0;
};

namespace {

// pool head: box table, runtime records and work tables for max_active slots
size_t head_size(int slots) {
  size_t b = align_up(sizeof(hydro::DevBox) * slots, ALIGN) + align_up(sizeof(hydro::BoxRt) * slots, ALIGN);
  size_t ints = 0;
  for (int t = 0; t < hydro::NTABLES; t++) {
    const int nslot = hydro::TABLE_PER_PRECISION[t] ? 2 : 1;
    ints += nslot * (2 * (size_t)slots * hydro::TABLE_ZDIM[t] + 1);
  }
  return b + align_up(ints * sizeof(int), ALIGN);
}

void fill_geometry(Request* r) {
  hydro::HostBox& hb = r->hb;
  hb.d = r->d;
  hb.pitch = (long long)align_up((size_t)(r->d.nx + 2 * HYDRO_NG), 4);
  hb.plane = hb.pitch * (r->d.ny + 2 * HYDRO_NG);
  hb.vs = (long long)align_up((size_t)(hb.plane * (r->d.nz + 2 * HYDRO_NG)), 32);
  hb.interior = (long long)r->d.nx * r->d.ny * r->d.nz;
  hb.active = true;
  r->state_bytes = align_up(5 * (size_t)hb.vs * sizeof(double), ALIGN);
  const size_t elem = r->d.precision == HYDRO_MIXED ? sizeof(float) : sizeof(double);
  r->work_bytes = align_up((size_t)hydro::NFIELDS * hb.vs * elem, ALIGN);
}

hydro::DevBox dev_box(const Request* r) {
  hydro::DevBox db;
  memset(&db, 0, sizeof db);
  const hydro::HostBox& hb = r->hb;
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
  db.stage_off = 0;
  const double dx[3] = {hb.d.dx, hb.d.dy, hb.d.dz};
  for (int a = 0; a < 3; a++) {
    db.dx[a] = dx[a];
    db.idx[a] = 1.0 / dx[a];
  }
  db.gamma = hb.d.gamma;
  db.igm1 = 1.0 / (hb.d.gamma - 1.0);
  db.gm1 = hb.d.gamma - 1.0;
  db.gamma_f = (float)db.gamma;
  db.igm1_f = (float)db.igm1;
  db.cfl = hb.d.cfl;
  for (int f = 0; f < 6; f++) db.bc[f] = hb.d.bc[f];
  return db;
}

// interior <-> ghosted state copies of one request (one 3D copy per variable)
cudaError_t copy_interior(hydro_server* s, Request* r, bool to_device, cudaStream_t st) {
  const hydro::HostBox& hb = r->hb;
  double* base = reinterpret_cast<double*>(s->pool) + hb.state_off;
  double* host = to_device ? r->ic.data() : r->result.data();
  const size_t nx = hb.d.nx, ny = hb.d.ny, nz = hb.d.nz;
  for (int v = 0; v < 5; v++) {
    cudaMemcpy3DParms p;
    memset(&p, 0, sizeof p);
    cudaPitchedPtr dev = make_cudaPitchedPtr(base + v * hb.vs, hb.pitch * sizeof(double), hb.pitch * sizeof(double),
                                             ny + 2 * HYDRO_NG);
    cudaPitchedPtr hst = make_cudaPitchedPtr(host + v * nx * ny * nz, nx * sizeof(double), nx * sizeof(double), ny);
    cudaPos dpos = make_cudaPos(HYDRO_NG * sizeof(double), HYDRO_NG, HYDRO_NG);
    p.extent = make_cudaExtent(nx * sizeof(double), ny, nz);
    if (to_device) {
      p.srcPtr = hst;
      p.dstPtr = dev;
      p.dstPos = dpos;
      p.kind = cudaMemcpyHostToDevice;
    } else {
      p.srcPtr = dev;
      p.srcPos = dpos;
      p.dstPtr = hst;
      p.kind = cudaMemcpyDeviceToHost;
    }
    cudaError_t e = cudaMemcpy3DAsync(&p, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Rebuilds the work tables of the resident set and copies them (and the box
// table) to the device on the compute stream, behind the previous tick, from a
// pinned staging buffer (pageable sources would make the host wait for the
// stream).
cudaError_t upload_plan(hydro_server* s) {
  hydro::Plan& p = s->plan;
  const int k = s->staging_next;
  s->staging_next ^= 1;
  cudaError_t e = cudaEventSynchronize(s->staging_ev[k]);  // the buffer's previous copies are done
  unsigned char* st = s->staging[k];
  const size_t dbytes = sizeof(hydro::DevBox) * p.nboxes;
  memcpy(st, s->dbox_host.data(), dbytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.dboxes, st, dbytes, cudaMemcpyHostToDevice, s->compute);
  p.has_fp64 = p.has_mixed = false;
  for (int b = 0; b < p.nboxes; b++)
    if (s->slots[b].active) (s->slots[b].d.precision == HYDRO_MIXED ? p.has_mixed : p.has_fp64) = true;
  int* ip = reinterpret_cast<int*>(st + align_up(dbytes, ALIGN));
  for (int t = 0; t < hydro::NTABLES && e == cudaSuccess; t++)
    for (int sl = 0; sl < 2 && e == cudaSuccess; sl++) {
      hydro::WorkTable& w = p.tab[t][sl];
      if (w.capacity == 0) continue;
      int* start = ip;
      int* item = ip + w.capacity + 1;
      ip += 2 * w.capacity + 1;
      w.nitems = hydro::build_table(p, t, sl, w.tpb, w.order, start, item);
      w.blocks = start[w.nitems];
      e = cudaMemcpyAsync(w.start, start, sizeof(int) * (w.nitems + 1), cudaMemcpyHostToDevice, s->compute);
      if (e == cudaSuccess && w.nitems)
        e = cudaMemcpyAsync(w.item, item, sizeof(int) * w.nitems, cudaMemcpyHostToDevice, s->compute);
    }
  if (e == cudaSuccess) e = cudaEventRecord(s->staging_ev[k], s->compute);
  return e;
}

void finish_request(hydro_server* s, Request* r, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->slot >= 0) {
    s->slots[r->slot].active = false;
    s->slot_req[r->slot] = nullptr;
    r->slot = -1;
  }
  if (r->state_bytes && r->state_off) s->mem.release(r->state_off - s->head_bytes, r->state_bytes + r->work_bytes);
  r->st = RS_DONE;
  if (r->status == HYDRO_OK) r->status = status;
  r->t_done = Clock::now();
  r->ic.clear();
  r->ic.shrink_to_fit();
  s->finished++;
  s->cv.notify_all();
}

// Admits queued requests (in submission order, later ones may pass a head
// that does not fit yet) while slots and memory allow.  Caller holds mu.
void admit(hydro_server* s, std::vector<Request*>* admitted) {
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    int slot = -1;
    for (int b = 0; b < s->plan.nboxes; b++)
      if (!s->slot_req[b] && !s->slots[b].active) {
        slot = b;
        break;
      }
    if (slot < 0) break;
    Request* r = *it;
    size_t off = 0;
    if (!s->mem.alloc(r->state_bytes + r->work_bytes, &off)) {
      ++it;
      continue;
    }
    off += s->head_bytes;
    r->state_off = off;
    r->hb.state_off = (long long)(off / sizeof(double));
    r->work_off = off + r->state_bytes;
    r->hb.work_off = (long long)r->work_off;
    r->slot = slot;
    r->st = RS_ACTIVE;
    r->t_admit = Clock::now();
    s->slot_req[slot] = r;
    s->slots[slot] = r->hb;
    s->dbox_host[slot] = dev_box(r);
    s->admitted++;
    admitted->push_back(r);
    it = s->queue.erase(it);
  }
}

// Host-only tick of a dry-run server: one step for every resident request.
void dry_tick(hydro_server* s) {
  std::vector<Request*> admitted, done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    admit(s, &admitted);
    for (Request* r : s->slot_req)
      if (r && ++r->steps_done >= r->nsteps) done.push_back(r);
    s->ticks++;
  }
  for (Request* r : s->slot_req)
    if (r && r->nsteps == 0 && std::find(done.begin(), done.end(), r) == done.end()) done.push_back(r);
  for (Request* r : done) {
    r->result = r->ic;
    r->steps = r->nsteps;
    finish_request(s, r, HYDRO_OK);
  }
}

int gpu_tick(hydro_server* s) {
  std::vector<Request*> admitted;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    admit(s, &admitted);
  }
  cudaError_t e = cudaSuccess;
  // uploads of the newly admitted requests on the copy stream
  for (Request* r : admitted) {
    if (e == cudaSuccess) e = copy_interior(s, r, true, s->copy);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->compute, r->ev, 0);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(s->plan.rt + r->slot, 0, sizeof(hydro::BoxRt), s->compute);
  }
  // requests that take no step finish as soon as they are resident
  std::vector<Request*> done_now;
  bool any_active = false;
  for (Request* r : s->slot_req) {
    if (!r || r->st != RS_ACTIVE) continue;
    if (r->nsteps == 0) done_now.push_back(r);
    else any_active = true;
  }
  for (Request* r : done_now) {
    s->slots[r->slot].active = false;
    memset(&s->dbox_host[r->slot], 0, sizeof(hydro::DevBox));
    r->st = RS_FINISHING;
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->compute);
    s->finishing.push_back(r);
  }
  if (e == cudaSuccess && (any_active || !admitted.empty() || !done_now.empty())) e = upload_plan(s);
  std::vector<Request*> finished_now;
  if (e == cudaSuccess && any_active) {
    for (int st = hydro::ST_FILL; st < hydro::NSTAGES && e == cudaSuccess; st++) {
      int n = 0;
      e = hydro::launch_stage(s->plan, static_cast<hydro::Stage>(st), s->compute, nullptr, nullptr,
                              st == hydro::ST_DT ? 1 : 0, &n);
      s->launches += n;
    }
    s->ticks++;
    for (Request* r : s->slot_req) {
      if (!r || r->st != RS_ACTIVE) continue;
      if (++r->steps_done >= r->nsteps) finished_now.push_back(r);
    }
    for (Request* r : finished_now) {
      // leaves the batch before the next tick (a zeroed box is skipped by the dt
      // stage, so its time and step count stay put); memory is freed after the copy-back
      s->slots[r->slot].active = false;
      memset(&s->dbox_host[r->slot], 0, sizeof(hydro::DevBox));
      r->st = RS_FINISHING;
      if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->compute);
    }
  }
  if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("server tick: ") + cudaGetErrorString(e));
  // copy back what finished on earlier ticks while this tick computes
  std::vector<Request*> keep;
  for (Request* r : s->finishing) {
    if (std::find(finished_now.begin(), finished_now.end(), r) != finished_now.end()) {
      keep.push_back(r);
      continue;
    }
    hydro::BoxRt rt;
    r->result.assign(5 * (size_t)r->hb.interior, 0.0);
    cudaError_t ce = cudaStreamWaitEvent(s->copy, r->ev, 0);
    if (ce == cudaSuccess) ce = copy_interior(s, r, false, s->copy);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(&rt, s->plan.rt + r->slot, sizeof rt, cudaMemcpyDeviceToHost, s->copy);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->copy);
    if (ce != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("server copy-back: ") + cudaGetErrorString(ce));
    r->steps = (int)rt.steps;
    r->time = rt.time;
    finish_request(s, r, rt.status ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK);
  }
  s->finishing = keep;
  for (Request* r : finished_now) s->finishing.push_back(r);
  return HYDRO_OK;
}

void worker_main(hydro_server* s) {
  if (!s->dry) cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool idle = s->queue.empty();
      for (Request* r : s->slot_req) idle = idle && !r;
      idle = idle && s->finishing.empty();
      if (idle) {
        if (s->stop) return;
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      if (s->stop && !s->worker_error.empty()) return;
    }
    if (s->dry) {
      dry_tick(s);
      continue;
    }
    if (gpu_tick(s) != HYDRO_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->worker_error = hydro_last_error();
      // fail everything that is still waiting; the server stops serving
      for (auto& kv : s->reqs)
        if (kv.second->st != RS_DONE) {
          kv.second->st = RS_DONE;
          kv.second->status = HYDRO_ERR_CUDA;
          kv.second->t_done = Clock::now();
        }
      s->queue.clear();
      s->cv.notify_all();
      return;
    }
  }
}

}  // namespace

extern "C" {

int hydro_server_create(const hydro_server_config* cfg, hydro_server** out) {
  if (!cfg || !out) return fail(HYDRO_ERR_INVALID, "null argument");
  *out = nullptr;
  if (cfg->max_active < 1 || cfg->max_active > 4096) return fail(HYDRO_ERR_INVALID, "max_active must be in [1, 4096]");
  const bool dry = cfg->dry_run != 0;
  if (!dry && !cfg->pool_dev) return fail(HYDRO_ERR_INVALID, "pool_dev is null (set dry_run for a host-only server)");
  if (reinterpret_cast<uintptr_t>(cfg->pool_dev) % ALIGN) return fail(HYDRO_ERR_INVALID, "pool must be 256-byte aligned");
  const size_t head = head_size(cfg->max_active);
  if (cfg->pool_bytes <= head) return fail(HYDRO_ERR_NOMEM, "pool smaller than the server's tables");
  std::unique_ptr<hydro_server> s(new hydro_server());
  s->cfg = *cfg;
  s->dry = dry;
  s->pool = static_cast<unsigned char*>(cfg->pool_dev);
  s->head_bytes = head;
  s->mem.reset(cfg->pool_bytes - head);
  const int n = cfg->max_active;
  s->slots.assign(n, hydro::HostBox());
  for (auto& hb : s->slots) {
    memset(&hb.d, 0, sizeof hb.d);
    hb.active = false;
  }
  s->slot_req.assign(n, nullptr);
  s->dbox_host.assign(n, hydro::DevBox());
  memset(s->dbox_host.data(), 0, sizeof(hydro::DevBox) * n);
  hydro::Plan& p = s->plan;
  p.nboxes = n;
  p.boxes = s->slots.data();
  if (!dry) {
    cudaError_t e = cudaGetDevice(&s->device);
    unsigned char* h = s->pool;
    p.dboxes = reinterpret_cast<hydro::DevBox*>(h);
    h += align_up(sizeof(hydro::DevBox) * n, ALIGN);
    p.rt = reinterpret_cast<hydro::BoxRt*>(h);
    h += align_up(sizeof(hydro::BoxRt) * n, ALIGN);
    int* ip = reinterpret_cast<int*>(h);
    for (int t = 0; t < hydro::NTABLES; t++)
      for (int sl = 0; sl < 2; sl++) {
        hydro::WorkTable& w = p.tab[t][sl];
        w.capacity = (sl == 0 || hydro::TABLE_PER_PRECISION[t]) ? n * hydro::TABLE_ZDIM[t] : 0;
        w.nitems = w.blocks = 0;
        w.tpb = hydro::default_tpb(t);
        w.order = 1;  // largest items first: uneven requests share every launch
        w.start = w.item = nullptr;
        if (w.capacity) {
          w.start = ip;
          ip += w.capacity + 1;
          w.item = ip;
          ip += w.capacity;
        }
      }
    p.state = reinterpret_cast<double*>(s->pool);
    p.work = s->pool;
    p.work_bytes = cfg->pool_bytes;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemset(s->pool, 0, head);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
      e = cudaHostAlloc(reinterpret_cast<void**>(&s->staging[k]), head, cudaHostAllocDefault);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->staging_ev[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      for (int k = 0; k < 2; k++) {
        if (s->staging[k]) cudaFreeHost(s->staging[k]);
        if (s->staging_ev[k]) cudaEventDestroy(s->staging_ev[k]);
      }
      if (s->compute) cudaStreamDestroy(s->compute);
      if (s->copy) cudaStreamDestroy(s->copy);
      return fail(HYDRO_ERR_CUDA, std::string("hydro_server_create: ") + cudaGetErrorString(e));
    }
  }
  hydro_server* raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return HYDRO_OK;
}

int hydro_server_destroy(hydro_server* s) {
  if (!s) return fail(HYDRO_ERR_INVALID, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Request* r : s->queue) {  // never admitted: cancelled
      r->st = RS_DONE;
      r->status = HYDRO_ERR_INVALID;
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (!s->dry) {
    cudaStreamSynchronize(s->compute);
    cudaStreamSynchronize(s->copy);
    for (auto& kv : s->reqs)
      if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    cudaStreamDestroy(s->compute);
    cudaStreamDestroy(s->copy);
    for (int k = 0; k < 2; k++) {
      cudaFreeHost(s->staging[k]);
      cudaEventDestroy(s->staging_ev[k]);
    }
  }
  delete s;
  return HYDRO_OK;
}

int hydro_submit(hydro_server* s, const hydro_request* r, int64_t* ticket) {
  if (!s || !r || !ticket) return fail(HYDRO_ERR_INVALID, "null argument");
  if (r->nsteps < 0) return fail(HYDRO_ERR_INVALID, "nsteps must be >= 0");
  if (!r->ic_host) return fail(HYDRO_ERR_INVALID, "null initial state");
  size_t sb = 0, wb = 0;
  if (hydro_workspace_size(&r->desc, 1, &sb, &wb) != HYDRO_OK) return HYDRO_ERR_INVALID;
  std::unique_ptr<Request> q(new Request());
  q->d = r->desc;
  q->nsteps = r->nsteps;
  fill_geometry(q.get());
  if (q->state_bytes + q->work_bytes > s->cfg.pool_bytes - s->head_bytes)
    return fail(HYDRO_ERR_NOMEM, "request larger than the server's memory budget");
  const size_t n = 5 * (size_t)q->hb.interior;
  q->ic.assign(r->ic_host, r->ic_host + n);
  if (!s->dry) {
    cudaError_t e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(HYDRO_ERR_CUDA, std::string("hydro_submit: ") + cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop || !s->worker_error.empty()) {
    if (q->ev) cudaEventDestroy(q->ev);
    return fail(HYDRO_ERR_INVALID, "server is stopping or failed: " + s->worker_error);
  }
  q->ticket = s->next_ticket++;
  q->t_submit = Clock::now();
  *ticket = q->ticket;
  s->queue.push_back(q.get());
  s->reqs[q->ticket] = std::move(q);
  s->cv.notify_all();
  return HYDRO_OK;
}

int hydro_poll(hydro_server* s, int64_t ticket, double* out_host, size_t out_bytes, hydro_result* info) {
  if (!s) return fail(HYDRO_ERR_INVALID, "null server");
  std::unique_ptr<Request> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(HYDRO_ERR_INVALID, "unknown ticket (or already collected)");
    Request* r = it->second.get();
    if (r->st != RS_DONE) return HYDRO_PENDING;
    const size_t need = r->result.size() * sizeof(double);
    if (out_host && out_bytes != need && r->status == HYDRO_OK)
      return fail(HYDRO_ERR_INVALID, "output size does not match the request's interior");
    done = std::move(it->second);
    s->reqs.erase(it);
  }
  Request* r = done.get();
  if (out_host && r->status == HYDRO_OK) memcpy(out_host, r->result.data(), r->result.size() * sizeof(double));
  if (info) {
    info->status = r->status;
    info->steps = r->steps;
    info->time = r->time;
    const bool admitted = r->t_admit.time_since_epoch().count() != 0;
    info->queued_s = admitted ? std::chrono::duration<double>(r->t_admit - r->t_submit).count() : 0.0;
    info->latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  }
  if (r->ev) cudaEventDestroy(r->ev);
  if (r->status != HYDRO_OK) return fail(r->status, "request failed");
  return HYDRO_OK;
}

int hydro_server_get_stats(hydro_server* s, hydro_server_stats* out) {
  if (!s || !out) return fail(HYDRO_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof *out);
  out->queued = (int64_t)s->queue.size();
  for (Request* r : s->slot_req) out->active += r != nullptr;
  out->finished = s->finished;
  out->admitted = s->admitted;
  out->ticks = s->ticks;
  out->kernel_launches = s->launches;
  out->bytes_in_use = (int64_t)s->mem.used();
  out->peak_bytes = (int64_t)s->mem.peak();
  out->budget_bytes = (int64_t)(s->cfg.pool_bytes - s->head_bytes);
  return HYDRO_OK;
}

}  // extern "C"
