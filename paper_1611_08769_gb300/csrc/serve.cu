// Serving loop: continuous (iteration-level) batching of encrypted FFTs.
//
// Clients submit requests (shape + host input ciphertexts + host output
// buffer) at any time. A worker thread owns one CUDA stream and repeats a
// tick: admit queued requests while the HBM budget has room (each request's
// ciphertexts -- scratch wires, inputs, outputs -- get one contiguous range
// of a device arena; its input ciphertexts are copied in), then launch, in
// one level launch, the next level of every active request, so requests that
// arrive while others run join at the next tick and share its launch; a
// request whose last level ran gets its output fix-ups and a copy back to the
// client's buffer, and its range is released once that copy completed.
//
// All requests share (n, ell); they may use different client keys because
// leveled GSW gates need no evaluation key. Each request's compiled program
// (cached per shape) has its references rewritten to absolute arena slots at
// admission, so gates of different requests mix freely in one launch.
#include <cuda_runtime.h>

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
#include <tuple>
#include <vector>

#include "common.h"
#include "netlist.h"
#include "plan.h"

namespace sfft {

namespace {

using Clock = std::chrono::steady_clock;

// Later requests that may be admitted past one that waits at the head of the
// queue for room.
constexpr uint32_t kMaxBypass = 16;

// First-fit allocator of ranges [0, capacity) with coalescing frees.
class RangeAlloc {
 public:
  void reset(uint64_t cap) {
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(uint64_t n, uint64_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<uint64_t, uint64_t> free_;   // offset -> length
};

struct Shape4 {
  uint32_t N1, N2, F, f;
  bool operator<(const Shape4& o) const {
    return std::tie(N1, N2, F, f) < std::tie(o.N1, o.N2, o.F, o.f);
  }
};

// A shape's compiled program: host copy (levels, counts) and device copy
// (descriptors, coefficients, fix-ups) that admission remaps on the device.
struct ShapeProgram {
  Program host;
  DeviceProgram dev;
  ~ShapeProgram() { free_device_program(&dev); }
};

struct Request {
  uint64_t ticket = 0;
  Shape4 shape{};
  const Program* prog = nullptr;
  const DeviceProgram* dprog = nullptr;
  uint32_t bypassed = 0;                   // later requests admitted while this one waited at the head
  const uint32_t* h_in = nullptr;
  uint32_t* h_out = nullptr;
  uint64_t base = 0, nslots = 0;          // arena range (ciphertexts)
  uint64_t dbase = 0, ndesc = 0;           // descriptor-pool range (gates)
  uint64_t fbase = 0, nfix = 0;            // fix-up pool range
  size_t level = 0;
  int state = 0;                           // 0 queued, 1 active, 2 copying out, 3 done
  cudaEvent_t done_ev = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

}  // namespace sfft

struct sfft_server {
  sfft::Shape s;
  uint32_t max_active = 64;
  uint64_t arena_cts = 0;
  uint32_t* arena = nullptr;
  sfft::RangeAlloc arena_alloc;
  // device descriptor pool (gates) and fix-up pool
  sfft::GateDesc* dpool = nullptr;
  sfft::GateAux* apool = nullptr;
  uint64_t dpool_cap = 0;
  sfft::RangeAlloc dpool_alloc;
  sfft::FixDesc* fpool = nullptr;
  uint64_t fpool_cap = 0;
  sfft::RangeAlloc fpool_alloc;
  // per-tick gathered level (written in stream order by the gather kernel);
  // tick_ev[k] marks the end of the last tick with parity k, so the host runs
  // at most two ticks ahead of the device
  sfft::GateDesc* tick_desc = nullptr;
  sfft::GateAux* tick_aux = nullptr;
  uint64_t tick_cap = 0;
  cudaEvent_t tick_ev[2] = {nullptr, nullptr};
  bool tick_ev_used[2] = {false, false};
  uint8_t* bx = nullptr;
  int* err = nullptr;
  cudaStream_t stream = nullptr;
  bool tc = false;
  uint32_t variant = 0;            // circuit variant flags of every request

  std::map<sfft::Shape4, std::unique_ptr<sfft::ShapeProgram>> programs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<sfft::Request>> queue;
  std::vector<std::shared_ptr<sfft::Request>> active;
  std::map<uint64_t, std::shared_ptr<sfft::Request>> by_ticket;
  uint64_t next_ticket = 1;
  bool stop = false;
  int worker_error = 0;
  std::string worker_msg;
  std::thread worker;
  // statistics
  uint64_t completed = 0, ticks = 0, tick_gates = 0, peak_active = 0;
  std::vector<double> latencies_ms;
};

namespace sfft {

namespace {

// A program-relative reference -> an absolute arena slot (region 0).
__host__ __device__ __forceinline__ uint32_t remap(uint32_t ref, uint64_t scr, uint64_t in, uint64_t out) {
  if (ref == REF_NONE) return ref;
  const uint32_t region = ref >> 30, slot = ref & SLOT_MASK;
  const uint64_t base = region == REG_SCRATCH ? scr : region == REG_IN ? in : out;
  return (uint32_t)(base + slot);   // region bits 0: the arena
}

// Admission: a request's descriptors and fix-ups, remapped to its arena range,
// written into its pool ranges (grid-stride over gates, then fix-ups).
__global__ void k_admit_remap(const GateDesc* src, const GateAux* asrc, uint64_t n, GateDesc* dst,
                              GateAux* adst, const FixDesc* fsrc, uint64_t nf, FixDesc* fdst,
                              uint64_t scr, uint64_t in, uint64_t out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
    const GateDesc d = src[g];
    dst[g] = GateDesc{remap(d.a, scr, in, out), remap(d.b, scr, in, out), remap(d.o0, scr, in, out),
                      remap(d.o1, scr, in, out)};
    adst[g] = asrc[g];
  }
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += stride) {
    FixDesc f = fsrc[k];
    f.dst = (uint32_t)(out + f.dst);   // absolute arena slot (REG_OUT base = arena)
    if (f.kind <= 1) f.src = remap(f.src, scr, in, out);
    fdst[k] = f;
  }
}

// A tick's level: up to kTickJobs contiguous descriptor runs (every active
// request's products, then their linear gates) gathered into the tick buffer
// by one launch; job j copies cnt[j] gates from pool index src[j] to dst[j].
constexpr uint32_t kTickJobs = 128;
struct TickJobs {
  uint32_t n, pad;
  uint64_t src[kTickJobs], dst[kTickJobs], cnt[kTickJobs];
};

__global__ void k_tick_gather(TickJobs jobs, const GateDesc* dpool, const GateAux* apool, GateDesc* tdesc,
                              GateAux* taux) {
  const uint32_t j = blockIdx.y;
  if (j >= jobs.n) return;
  const uint64_t cnt = jobs.cnt[j], src = jobs.src[j], dst = jobs.dst[j];
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cnt;
       g += (uint64_t)gridDim.x * blockDim.x) {
    tdesc[dst + g] = dpool[src + g];
    taux[dst + g] = apool[src + g];
  }
}

// Admission (under the lock): arena and pool ranges, then, on the server
// stream, the device remap of the shape's program into the pools and the copy
// of the client's inputs (h_in stays valid until the request's wait returns,
// so nothing here waits for the copies).
int admit(sfft_server* sv, Request* r) {
  const Program& p = *r->prog;
  r->nslots = p.scratch_slots + p.n_inputs + p.n_outputs;
  if (!sv->arena_alloc.alloc(r->nslots, &r->base)) return 1;   // no room yet
  r->ndesc = p.desc.size();
  if (r->ndesc && !sv->dpool_alloc.alloc(r->ndesc, &r->dbase)) {
    sv->arena_alloc.release(r->base, r->nslots);
    return 1;
  }
  r->nfix = p.fix.size();
  if (r->nfix && !sv->fpool_alloc.alloc(r->nfix, &r->fbase)) {
    sv->arena_alloc.release(r->base, r->nslots);
    if (r->ndesc) sv->dpool_alloc.release(r->dbase, r->ndesc);
    return 1;
  }
  const uint64_t scr = r->base, in = r->base + p.scratch_slots, out = in + p.n_inputs;
  cudaStream_t st = sv->stream;
  const uint64_t work = std::max<uint64_t>(r->ndesc, r->nfix);
  if (work) {
    const unsigned blocks = (unsigned)std::min<uint64_t>((work + 255) / 256, 1024);
    k_admit_remap<<<blocks, 256, 0, st>>>(r->dprog->desc, r->dprog->aux, r->ndesc, sv->dpool + r->dbase,
                                          sv->apool + r->dbase, r->dprog->fix, r->nfix,
                                          sv->fpool + r->fbase, scr, in, out);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sv->arena + in * sv->s.ctw, r->h_in, p.n_inputs * sv->s.ctw * 4,
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "server admission");
  r->level = 0;
  r->state = 1;
  r->t_admit = Clock::now();
  return 0;
}

int ensure_tick_capacity(sfft_server* sv, uint64_t n) {
  if (n <= sv->tick_cap) return SFFT_OK;
  cudaStreamSynchronize(sv->stream);   // the old buffers may still be read
  cudaFree(sv->tick_desc);
  cudaFree(sv->tick_aux);
  uint64_t cap = std::max<uint64_t>(n, 2 * sv->tick_cap);
  cudaError_t e = cudaMalloc((void**)&sv->tick_desc, cap * sizeof(GateDesc));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->tick_aux, cap * sizeof(GateAux));
  if (e != cudaSuccess) return cuda_fail(e, "tick buffer");
  sv->tick_cap = cap;
  return SFFT_OK;
}

// One tick (worker thread, lock not held): the next level of every active
// request, gathered on the device by one launch and evaluated by one launch
// of products (and one of linear gates).
int tick(sfft_server* sv, std::vector<std::shared_ptr<Request>>& act) {
  cudaStream_t st = sv->stream;
  // the level's products of every active request, then their linear gates
  uint64_t n = 0, nprod = 0;
  for (auto& r : act) {
    const Program& p = *r->prog;
    if (r->level + 1 >= p.level_off.size()) continue;
    n += p.level_off[r->level + 1] - p.level_off[r->level];
    nprod += p.lin_start[r->level] - p.level_off[r->level];
  }
  int rc = ensure_tick_capacity(sv, n);
  if (rc) return rc;
  TickJobs jobs;
  jobs.n = 0;
  jobs.pad = 0;
  uint64_t at[2] = {0, nprod}, most = 0;
  for (int ph = 0; ph < 2; ph++) {
    for (auto& r : act) {
      const Program& p = *r->prog;
      if (r->level + 1 >= p.level_off.size()) continue;
      const uint64_t cut[3] = {p.level_off[r->level], p.lin_start[r->level], p.level_off[r->level + 1]};
      const uint64_t cnt = cut[ph + 1] - cut[ph];
      if (!cnt) continue;
      if (jobs.n == kTickJobs) return fail(SFFT_EINVAL, "too many descriptor runs in one tick");
      jobs.src[jobs.n] = r->dbase + cut[ph];
      jobs.dst[jobs.n] = at[ph];
      jobs.cnt[jobs.n] = cnt;
      jobs.n++;
      at[ph] += cnt;
      most = std::max(most, cnt);
    }
  }
  for (auto& r : act)
    if (r->level + 1 < r->prog->level_off.size()) r->level++;
  if (jobs.n) {
    const dim3 grid((unsigned)std::min<uint64_t>((most + 255) / 256, 64), jobs.n);
    k_tick_gather<<<grid, 256, 0, st>>>(jobs, sv->dpool, sv->apool, sv->tick_desc, sv->tick_aux);
    count_launches(1);
  }
  if (n) {
    KArgs a = make_args(sv->s);
    a.desc = sv->tick_desc;
    a.aux = sv->tick_aux;
    a.n = nprod;
    a.base[REG_SCRATCH] = sv->arena;
    a.base[REG_IN] = sv->arena;
    a.base[REG_OUT] = sv->arena;
    a.err = sv->err;
    a.kernel = KERNEL_AUTO;
    a.bx = sv->bx;
    if ((rc = launch_gates(a, st))) return rc;
    a.desc = sv->tick_desc + nprod;
    a.aux = sv->tick_aux + nprod;
    a.n = n - nprod;
    if ((rc = launch_linear(a, st))) return rc;
  }
  sv->ticks++;
  sv->tick_gates += n;
  // finished requests: fix-ups, copy out, completion event
  for (auto& r : act) {
    const Program& p = *r->prog;
    if (r->state != 1 || r->level + 1 < p.level_off.size()) continue;
    if (r->nfix) {
      KArgs a = make_args(sv->s);
      a.base[REG_SCRATCH] = sv->arena;
      a.base[REG_IN] = sv->arena;
      a.base[REG_OUT] = sv->arena;
      if ((rc = launch_fixups(sv->fpool + r->fbase, r->nfix, a, st))) return rc;
    }
    const uint64_t out = r->base + p.scratch_slots + p.n_inputs;
    cudaMemcpyAsync(r->h_out, sv->arena + out * sv->s.ctw, p.n_outputs * sv->s.ctw * 4,
                    cudaMemcpyDeviceToHost, st);
    cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
    cudaEventRecord(r->done_ev, st);
    r->state = 2;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "server tick");
}

void worker_main(sfft_server* sv) {
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // admission in arrival order; a request that does not fit yet is passed
    // by later ones that do, until kMaxBypass of them have passed it, after
    // which nothing is admitted before it (no starvation of large requests)
    for (auto it = sv->queue.begin(); it != sv->queue.end() && sv->active.size() < sv->max_active;) {
      const bool head = it == sv->queue.begin();
      auto r = *it;
      const int rc = admit(sv, r.get());
      if (rc < 0) {
        sv->worker_error = rc;
        sv->worker_msg = sfft_last_error();
        sv->stop = true;
        break;
      }
      if (rc == 1) {
        if (head && r->bypassed >= kMaxBypass) break;
        ++it;
        continue;
      }
      if (!head) sv->queue.front()->bypassed++;
      sv->active.push_back(r);
      it = sv->queue.erase(it);
    }
    sv->peak_active = std::max<uint64_t>(sv->peak_active, sv->active.size());
    // completions
    bool progressed = false;
    for (size_t k = 0; k < sv->active.size();) {
      auto& r = sv->active[k];
      if (r->state == 2 && cudaEventQuery(r->done_ev) == cudaSuccess) {
        cudaEventDestroy(r->done_ev);
        r->done_ev = nullptr;
        r->t_done = Clock::now();
        r->state = 3;
        sv->arena_alloc.release(r->base, r->nslots);
        if (r->ndesc) sv->dpool_alloc.release(r->dbase, r->ndesc);
        if (r->nfix) sv->fpool_alloc.release(r->fbase, r->nfix);
        sv->completed++;
        sv->latencies_ms.push_back(
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        sv->active.erase(sv->active.begin() + k);
        progressed = true;
      } else {
        k++;
      }
    }
    if (progressed) sv->cv_done.notify_all();
    if (sv->stop && sv->active.empty()) break;
    if (sv->stop && sv->worker_error) break;
    std::vector<std::shared_ptr<Request>> running;
    for (auto& r : sv->active)
      if (r->state == 1) running.push_back(r);
    if (running.empty()) {
      if (sv->active.empty())
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
      else
        sv->cv_work.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    lk.unlock();
    // at most two ticks in flight: wait for the tick before last
    const int k = (int)(sv->ticks & 1);
    if (sv->tick_ev_used[k]) cudaEventSynchronize(sv->tick_ev[k]);
    const int rc = tick(sv, running);
    cudaEventRecord(sv->tick_ev[k], sv->stream);
    sv->tick_ev_used[k] = true;
    lk.lock();
    if (rc) {
      sv->worker_error = rc;
      sv->worker_msg = sfft_last_error();
      sv->stop = true;
    }
  }
  sv->cv_done.notify_all();
}

}  // namespace

}  // namespace sfft

using namespace sfft;

extern "C" {

int sfft_server_create(const sfft_params* p, uint64_t hbm_budget_bytes, uint32_t max_active,
                       uint32_t flags, sfft_server** out) {
  if (!out) return fail(SFFT_EINVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<sfft_server> sv(new (std::nothrow) sfft_server);
  if (!sv) return fail(SFFT_ENOMEM, "host allocation failed");
  int rc = make_shape(p, &sv->s, false);
  if (rc) return rc;
  sv->max_active = max_active ? max_active : 64;
  sv->variant = flags & (SFFT_PLAN_XCARRY | SFFT_PLAN_NAND | SFFT_PLAN_ENC_TWIDDLE);
  if (!Circuit().set_variant(sv->variant))
    return fail(SFFT_EINVAL, "SFFT_PLAN_XCARRY and SFFT_PLAN_NAND are exclusive");
  const uint64_t ctb = sv->s.ctw * 4;
  KArgs k = make_args(sv->s);
  sv->tc = gate_kernel_for(k) == KERNEL_TC;   // needs the B expansion region
  const uint64_t bx_bytes = sv->tc ? tc_bx_bytes(k, ~0ull >> 8) : 0;
  if (hbm_budget_bytes < bx_bytes + 64 * ctb) return fail(SFFT_EINVAL, "HBM budget too small");
  sv->arena_cts = (hbm_budget_bytes - bx_bytes) / ctb;
  cudaError_t e = cudaMalloc((void**)&sv->arena, sv->arena_cts * ctb);
  if (e != cudaSuccess) return fail(SFFT_ENOMEM, std::string("arena: ") + cudaGetErrorString(e));
  sv->arena_alloc.reset(sv->arena_cts);
  sv->dpool_cap = 1ull << 25;   // 32 Mi gates of descriptors (768 MB)
  sv->fpool_cap = 1ull << 20;
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->dpool, sv->dpool_cap * sizeof(GateDesc));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->apool, sv->dpool_cap * sizeof(GateAux));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->fpool, sv->fpool_cap * sizeof(FixDesc));
  if (e == cudaSuccess && bx_bytes) e = cudaMalloc((void**)&sv->bx, bx_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(sv->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    e = cudaEventCreateWithFlags(&sv->tick_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFree(sv->arena);
    cudaFree(sv->dpool);
    cudaFree(sv->apool);
    cudaFree(sv->fpool);
    cudaFree(sv->bx);
    cudaFree(sv->err);
    return fail(SFFT_ENOMEM, std::string("server buffers: ") + cudaGetErrorString(e));
  }
  sv->dpool_alloc.reset(sv->dpool_cap);
  sv->fpool_alloc.reset(sv->fpool_cap);
  sfft_server* raw = sv.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return SFFT_OK;
}

}  // extern "C"

namespace {

// The shape's compiled program, compiled on first use without holding the
// server's lock (a large circuit takes seconds on the host; the worker keeps
// ticking meanwhile). On return the lock is held.
int shape_program(sfft_server* sv, const sfft_request* req, std::unique_lock<std::mutex>& lk,
                  ShapeProgram** out) {
  const Shape4 shape{req->N1, req->N2, req->F, req->f};
  lk.lock();
  auto it = sv->programs.find(shape);
  if (it != sv->programs.end()) {
    *out = it->second.get();
    return SFFT_OK;
  }
  lk.unlock();
  Circuit c;
  c.set_variant(sv->variant);
  if (!build_fft(&c, req->N1, req->N2, req->F, req->f)) {
    lk.lock();
    return fail(SFFT_EINVAL, "invalid FFT shape");
  }
  std::unique_ptr<ShapeProgram> prog(new ShapeProgram);
  compile(c, sv->s, &prog->host);
  int rc = prog->host.noise_ok ? SFFT_OK : fail(SFFT_EPARAM, "static noise bound reaches q/4 for this shape");
  if (!rc) rc = make_device_program(prog->host, &prog->dev);
  lk.lock();
  if (rc) return rc;
  it = sv->programs.find(shape);   // another thread may have compiled it meanwhile
  if (it == sv->programs.end()) it = sv->programs.emplace(shape, std::move(prog)).first;
  *out = it->second.get();
  return SFFT_OK;
}

}  // namespace

extern "C" {

int sfft_server_prepare(sfft_server* sv, const sfft_request* req) {
  if (!sv || !req) return fail(SFFT_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(sv->mu, std::defer_lock);
  ShapeProgram* sp = nullptr;
  return shape_program(sv, req, lk, &sp);
}

int sfft_server_submit(sfft_server* sv, const sfft_request* req, const uint32_t* h_in, uint32_t* h_out,
                       uint64_t* ticket) {
  if (!sv || !req || !h_in || !h_out || !ticket) return fail(SFFT_EINVAL, "null argument");
  const Shape4 shape{req->N1, req->N2, req->F, req->f};
  std::unique_lock<std::mutex> lk(sv->mu, std::defer_lock);
  ShapeProgram* sprog = nullptr;
  const int rc = shape_program(sv, req, lk, &sprog);
  if (rc) return rc;
  if (sv->worker_error) return fail(sv->worker_error, "server stopped: " + sv->worker_msg);
  const Program* p = &sprog->host;
  if (p->scratch_slots + p->n_inputs + p->n_outputs > sv->arena_cts || p->desc.size() > sv->dpool_cap)
    return fail(SFFT_ENOMEM, "request larger than the whole HBM budget");
  auto r = std::make_shared<Request>();
  r->ticket = sv->next_ticket++;
  r->shape = shape;
  r->prog = p;
  r->dprog = &sprog->dev;
  r->h_in = h_in;
  r->h_out = h_out;
  r->t_submit = Clock::now();
  sv->queue.push_back(r);
  sv->by_ticket[r->ticket] = r;
  *ticket = r->ticket;
  sv->cv_work.notify_one();
  return SFFT_OK;
}

int sfft_server_wait(sfft_server* sv, uint64_t ticket, uint32_t timeout_ms, double* latency_ms) {
  if (!sv) return fail(SFFT_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->by_ticket.find(ticket);
  if (it == sv->by_ticket.end()) return fail(SFFT_ENOTFOUND, "unknown ticket");
  auto r = it->second;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                       [&] { return r->state == 3 || sv->worker_error; });
  if (sv->worker_error) return fail(sv->worker_error, "server stopped: " + sv->worker_msg);
  if (!ok) return fail(SFFT_ETIMEOUT, "request not finished within the timeout");
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  sv->by_ticket.erase(it);
  return SFFT_OK;
}

int sfft_server_get_stats(sfft_server* sv, sfft_server_stats* st) {
  if (!sv || !st) return fail(SFFT_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  std::memset(st, 0, sizeof(*st));
  st->completed = sv->completed;
  st->queued = sv->queue.size();
  st->active = sv->active.size();
  st->ticks = sv->ticks;
  st->tick_gates = sv->tick_gates;
  st->peak_active = sv->peak_active;
  std::vector<double> l = sv->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    st->p50_ms = l[(l.size() - 1) / 2];
    st->p99_ms = l[std::min(l.size() - 1, (size_t)(0.99 * (l.size() - 1) + 0.5))];
    st->max_ms = l.back();
  }
  return SFFT_OK;
}

void sfft_server_free(sfft_server* sv) {
  if (!sv) return;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  cudaStreamSynchronize(sv->stream);
  for (auto& kv : sv->by_ticket)
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
  cudaFree(sv->arena);
  cudaFree(sv->dpool);
  cudaFree(sv->apool);
  cudaFree(sv->fpool);
  cudaFree(sv->tick_desc);
  cudaFree(sv->tick_aux);
  cudaFree(sv->bx);
  cudaFree(sv->err);
  for (cudaEvent_t ev : sv->tick_ev)
    if (ev) cudaEventDestroy(ev);
  sv->programs.clear();   // device copies of the shape programs
  cudaStreamDestroy(sv->stream);
  delete sv;
}

}  // extern "C"
