// Request server of libpmf (declared in include/pmf.h, "Serving"): resident
// filters of mixed dimension, per-filter request queues, continuous batching
// onto three streams, admission under a device-memory budget.
//
// Host loop (pmf_server_replay): requests are released at their arrival time
// into their filter's queue; a filter with a queued request and nothing on the
// device is "ready".  Whenever fewer than PMF_SERVE_INFLIGHT batches are in
// flight, every ready filter contributes its head request to the next batch:
// 1-D items -> one launch of the 1-D kernel, 2-D items -> one launch of the
// fused batch kernel (each with its item array and per-item time constants in
// one copy), 3-D items -> their pipelines.  Completed batches (events, checked
// in order) release their filters; a request completes after its last chunk.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pmf.h"
#include "pmf_internal.cuh"
#include "pmf_model.cuh"
#include "pmf_tc.cuh"

using namespace pmf;

namespace {

constexpr int kInflight = PMF_SERVE_INFLIGHT;
constexpr int kMaxBatch = 4096;   // items per batch and dimension

// Fixed pool of host threads for the per-item time-update constants.
class Pool {
 public:
  explicit Pool(int workers) {
    for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  // f(i) for i in [0, n); the caller works too and returns when all are done
  void run(int n, const std::function<void(int)>& f) {
    if (n <= 0) return;
    auto job = std::make_shared<Job>();
    job->f = &f;
    job->n = n;
    if (n > 8 && !th_.empty()) {
      {
        std::lock_guard<std::mutex> g(mu_);
        job_ = job;
        ++gen_;
      }
      cv_.notify_all();
    }
    work(*job);
    while (job->done.load(std::memory_order_acquire) < n) std::this_thread::yield();
    std::lock_guard<std::mutex> g(mu_);
    if (job_ == job) job_.reset();
  }

 private:
  struct Job {
    const std::function<void(int)>* f = nullptr;
    int n = 0;
    std::atomic<int> next{0}, done{0};
  };
  static void work(Job& j) {
    for (;;) {
      const int i = j.next.fetch_add(1);
      if (i >= j.n) return;
      (*j.f)(i);
      j.done.fetch_add(1, std::memory_order_release);
    }
  }
  void loop() {
    long long seen = 0;
    for (;;) {
      std::shared_ptr<Job> j;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        j = job_;
      }
      if (j) work(*j);
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::shared_ptr<Job> job_;
  long long gen_ = 0;
  bool stop_ = false;
};

struct SFilter {
  bool alive = false;
  pmf_config cfg{};
  MeasParams mp{};         // model; z per request
  long long P = 0, bytes = 0;
  DevState* st = nullptr;
  float* buf = nullptr;    // 2 P floats
  MeasParams* d_mp = nullptr;
  TcTables tct{};          // 2-D/3-D: shared tables (owned by the server)
  void* tc3 = nullptr;     // 3-D pipeline state (owned)
  void* plan = nullptr;    // 2-D: the batch front kernel's results (owned)
  int cls = 128;           // 2-D: size class of its transform kernel
  // request in progress
  bool busy = false;
  long long cur = -1;
  double rem = 0.0;        // time update still to run for `cur`
  bool meas_pending = false;
  std::deque<long long> queue;
};

struct Flight {
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool used[3] = {false, false, false};
  std::vector<int> filters;
  StepItem* h_items[2] = {nullptr, nullptr};     // [0] 1-D, [1] 2-D (pinned)
  TimeConsts* h_tc[2] = {nullptr, nullptr};
  StepItem* d_items[2] = {nullptr, nullptr};
  TimeConsts* d_tc[2] = {nullptr, nullptr};
  Tc3Stage stage3{};                             // 3-D descriptors of this batch
  bool inflight = false;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct pmf_server {
  size_t budget = 0;
  int cap = 0, precision = 0;
  std::vector<SFilter> f;
  std::vector<int> free_ids;
  long long bytes = 0;
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};   // 1-D, 2-D, 3-D
  Slot1* d_slots1 = nullptr;
  FilterSlot* d_slots2 = nullptr;
  double* d_partials = nullptr;   // prior moments at admission
  double* d_aux = nullptr;
  std::map<long long, void*> tables;          // (kind, N) -> device table
  std::map<long long, size_t> hart_bytes;
  Flight ring[kInflight];
  int head = 0, tail = 0, inflight = 0;
  std::deque<int> ready;
  std::vector<char> in_ready;
  std::unique_ptr<Pool> pool;
  long long launches = 0, batches = 0, items = 0, max_batch = 0;
  std::string err;
};

namespace {

int sfail(pmf_server* s, int code, const std::string& msg) {
  s->err = msg;
  return code;
}

void free_filter(pmf_server* s, SFilter& f) {
  cudaFree(f.st);
  cudaFree(f.buf);
  cudaFree(f.d_mp);
  cudaFree(f.plan);
  tc3_free(f.tc3);
  s->bytes -= f.bytes;
  f = SFilter{};
}

int sync_all(pmf_server* s) {
  for (int k = 0; k < 3; ++k)
    if (cudaStreamSynchronize(s->s[k]) != cudaSuccess) return PMF_ERR_CUDA;
  return PMF_OK;
}

// Precision of a filter of n axes in the server: 1-D filters run the float32
// kernel (its table has no precision); 3-D filters of a BF16X6 server run
// FP16X3, the other split format within 1e-5 (the 3-D pipelines hold two
// operand planes).
int filter_precision(const pmf_server* s, int n) {
  return n == 1 || (n == 3 && s->precision == PMF_PREC_BF16X6) ? PMF_PREC_FP16X3 : s->precision;
}

// Shared device table of an axis size: kind 1 = 1-D kernel table, 2 = split
// Hartley planes + sinc table of the tensor-core kernels (size class 128),
// 3 and 4 = the same for the size-64 and size-96 classes of the batched 2-D
// kernels, 5 = the class-128 table in FP16X3 for the 3-D filters of a BF16X6
// server.  Adds new bytes to *add.
int table_for(pmf_server* s, int kind, int N, void** out, size_t* hb, long long* add, bool create) {
  const long long key = (long long)kind * 100000 + N;
  auto it = s->tables.find(key);
  if (it != s->tables.end()) {
    *out = it->second;
    if (hb) *hb = s->hart_bytes[key];
    return PMF_OK;
  }
  const int cls = kind == 3 ? 64 : kind == 4 ? 96 : 128;
  const int prec = kind == 5 ? PMF_PREC_FP16X3 : s->precision;
  const long long nb = kind == 1 ? (long long)tc1_table_bytes(N) : (long long)tc_axis_table_bytes(N, prec, cls);
  *add += nb;
  if (!create) return PMF_OK;
  void* t = nullptr;
  size_t h = 0;
  const int rc = kind == 1 ? tc1_build_table(N, &t) : tc_build_axis_table(N, prec, &t, &h, cls);
  if (rc) {
    cudaFree(t);
    return rc;
  }
  s->tables[key] = t;
  s->hart_bytes[key] = h;
  *out = t;
  if (hb) *hb = h;
  return PMF_OK;
}

// Put filter id on the ready list if it has work and nothing on the device.
void mark_ready(pmf_server* s, int id) {
  SFilter& f = s->f[id];
  if (f.busy || s->in_ready[id] || (f.cur < 0 && f.queue.empty())) return;
  s->in_ready[id] = 1;
  s->ready.push_back(id);
}

// Form and launch one batch from the ready filters.
int launch_batch(pmf_server* s, const double* z, const double* taus) {
  Flight& b = s->ring[s->head];
  b.filters.clear();
  for (int k = 0; k < 3; ++k) b.used[k] = false;
  struct Item {
    int id, kind, flags;
    double tau;
    long long req;
  };
  std::vector<Item> its;
  int count[3] = {0, 0, 0};
  std::deque<int> keep;
  while (!s->ready.empty()) {
    const int id = s->ready.front();
    s->ready.pop_front();
    SFilter& f = s->f[id];
    const int kind = f.cfg.nx - 1;
    if (kind < 2 && count[kind] >= kMaxBatch) {
      keep.push_back(id);
      continue;
    }
    s->in_ready[id] = 0;
    if (f.cur < 0) {
      f.cur = f.queue.front();
      f.queue.pop_front();
      f.rem = taus[f.cur];
      f.meas_pending = true;
    }
    const double tmax = MAXL * f.cfg.dt_sub * (1.0 - 1e-12);
    double tau = f.rem;
    if (tau > tmax) tau = tmax;
    f.rem -= tau;
    if (f.rem < 1e-12 * tmax) f.rem = 0.0;
    const int flags = (f.meas_pending ? 1 : 0) | (tau > 0.0 ? 2 : 0);
    its.push_back(Item{id, kind, flags, tau, f.cur});
    f.meas_pending = false;
    f.busy = true;
    ++count[kind];
    b.filters.push_back(id);
  }
  for (int id : keep) s->ready.push_back(id);
  if (its.empty()) return PMF_OK;

  // host constants (parallel), items
  std::vector<TimeConsts> tc3(its.size());
  // 2-D items: size class 128 first, then 96, then 64 (one transform kernel per range)
  auto cls2 = [&](int id) { return s->f[id].cls; };
  int n128 = 0, n96 = 0;
  for (const Item& it : its)
    if (it.kind == 1) {
      const int c = cls2(it.id);
      n128 += c == 128;
      n96 += c == 96;
    }
  int slot[2] = {0, 0}, slot96 = n128, slot64 = n128 + n96;
  std::vector<int> pos(its.size());
  for (size_t i = 0; i < its.size(); ++i) {
    const int k = its[i].kind;
    if (k != 1) {
      pos[i] = k == 0 ? slot[0]++ : 0;
      continue;
    }
    const int c = cls2(its[i].id);
    pos[i] = c == 128 ? slot[1]++ : c == 96 ? slot96++ : slot64++;
  }
  std::atomic<int> bad{0};
  const std::function<void(int)> fill = [&](int i) {
    const Item& it = its[i];
    SFilter& f = s->f[it.id];
    TimeConsts* dst = it.kind < 2 ? &b.h_tc[it.kind][pos[i]] : &tc3[i];
    if (it.tau > 0.0) {
      std::string why;
      if (time_consts(f.cfg, it.tau, dst, &why)) bad.store(1);
    }
    if (it.kind < 2) {
      StepItem& si = b.h_items[it.kind][pos[i]];
      si.slot = it.id;
      si.flags = it.flags;
      for (int j = 0; j < PMF_MAX_NZ; ++j) si.z[j] = (it.flags & 1) ? z[it.req * PMF_MAX_NZ + j] : 0.0;
    }
  };
  s->pool->run((int)its.size(), fill);
  if (bad.load()) return sfail(s, PMF_ERR_ARG, "time-update constants");

  // 1-D and 2-D: items and constants in one copy each, one launch each
  for (int k = 0; k < 2; ++k) {
    const int n = count[k];
    if (!n) continue;
    if (cudaMemcpyAsync(b.d_items[k], b.h_items[k], sizeof(StepItem) * n, cudaMemcpyHostToDevice, s->s[k]) !=
            cudaSuccess ||
        cudaMemcpyAsync(b.d_tc[k], b.h_tc[k], sizeof(TimeConsts) * n, cudaMemcpyHostToDevice, s->s[k]) !=
            cudaSuccess)
      return sfail(s, PMF_ERR_CUDA, "batch copies");
    s->launches += k == 0 ? tc1_batch_step(s->d_slots1, b.d_items[0], b.d_tc[0], n, s->s[0])
                          : tc_batch_epoch(s->precision, s->d_slots2, b.d_items[1], n, n128, n96, s->s[1], b.d_tc[1]);
    cudaEventRecord(b.ev[k], s->s[k]);
    b.used[k] = true;
  }
  // 3-D: every stage of the pipelines one launch over all the batch's 3-D filters
  if (count[2]) {
    std::vector<MeasParams> mps(count[2]);
    std::vector<Tc3Item> t3;
    t3.reserve(count[2]);
    for (size_t i = 0; i < its.size(); ++i) {
      const Item& it = its[i];
      if (it.kind != 2) continue;
      SFilter& f = s->f[it.id];
      MeasParams& mp = mps[t3.size()];
      mp = f.mp;
      for (int j = 0; j < PMF_MAX_NZ; ++j) mp.z[j] = z[it.req * PMF_MAX_NZ + j];
      Dims d{};
      d.nx = 3;
      d.P = f.P;
      for (int a = 0; a < 3; ++a) d.N[a] = f.cfg.N[a];
      t3.push_back(Tc3Item{f.tc3, d, &f.tct, (it.flags & 1) ? &mp : nullptr, (it.flags & 2) ? &tc3[i] : nullptr,
                           f.st, f.buf, f.buf + f.P});
    }
    const int r = tc3_batch(t3.data(), (int)t3.size(), filter_precision(s, 3), &b.stage3, s->s[2]);
    if (r < 0) return sfail(s, -r, "3-D batch");
    s->launches += r;
    cudaEventRecord(b.ev[2], s->s[2]);
    b.used[2] = true;
  }
  if (cudaGetLastError() != cudaSuccess) return sfail(s, PMF_ERR_CUDA, "batch launch");
  b.inflight = true;
  s->head = (s->head + 1) % kInflight;
  ++s->inflight;
  ++s->batches;
  s->items += (long long)its.size();
  if ((long long)its.size() > s->max_batch) s->max_batch = (long long)its.size();
  return PMF_OK;
}

// Retire finished batches in launch order; returns requests completed.
long long poll(pmf_server* s, double t0, const double* t_arrival, double* latency) {
  long long done = 0;
  while (s->inflight > 0) {
    Flight& b = s->ring[s->tail];
    bool ready = true;
    for (int k = 0; k < 3 && ready; ++k)
      if (b.used[k] && cudaEventQuery(b.ev[k]) != cudaSuccess) ready = false;
    if (!ready) break;
    const double t = now_s() - t0;
    for (int id : b.filters) {
      SFilter& f = s->f[id];
      f.busy = false;
      if (f.rem <= 0.0) {
        if (latency) latency[f.cur] = t - t_arrival[f.cur];
        f.cur = -1;
        ++done;
      }
      mark_ready(s, id);
    }
    b.inflight = false;
    s->tail = (s->tail + 1) % kInflight;
    --s->inflight;
  }
  return done;
}

}  // namespace

extern "C" {

int pmf_server_create(pmf_server** out, size_t hbm_budget, int max_filters, int precision) {
  if (!out || max_filters < 1 || max_filters > (1 << 24)) return PMF_ERR_ARG;
  if (precision != PMF_PREC_FP16X3 && precision != PMF_PREC_BF16X3 && precision != PMF_PREC_BF16X6 &&
      precision != PMF_PREC_TF32)
    return PMF_ERR_ARG;
  *out = nullptr;
  pmf_server* s = new (std::nothrow) pmf_server();
  if (!s) return PMF_ERR_OOM;
  s->budget = hbm_budget;
  s->cap = max_filters;
  s->precision = precision;
  s->f.resize(max_filters);
  s->in_ready.assign(max_filters, 0);
  for (int i = max_filters - 1; i >= 0; --i) s->free_ids.push_back(i);
  bool ok = true;
  for (int k = 0; k < 3; ++k) ok = ok && cudaStreamCreateWithFlags(&s->s[k], cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_slots1, sizeof(Slot1) * max_filters) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_slots2, sizeof(FilterSlot) * max_filters) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_partials, sizeof(double) * kMomentSlots * 4096) == cudaSuccess;
  ok = ok && cudaMalloc(&s->d_aux, sizeof(double) * kAuxSize) == cudaSuccess;
  for (int r = 0; r < kInflight && ok; ++r) {
    Flight& b = s->ring[r];
    for (int k = 0; k < 3 && ok; ++k) ok = cudaEventCreateWithFlags(&b.ev[k], cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
      ok = cudaMallocHost((void**)&b.h_items[k], sizeof(StepItem) * kMaxBatch) == cudaSuccess &&
           cudaMallocHost((void**)&b.h_tc[k], sizeof(TimeConsts) * kMaxBatch) == cudaSuccess &&
           cudaMalloc((void**)&b.d_items[k], sizeof(StepItem) * kMaxBatch) == cudaSuccess &&
           cudaMalloc((void**)&b.d_tc[k], sizeof(TimeConsts) * kMaxBatch) == cudaSuccess;
    }
  }
  if (!ok) {
    pmf_server_destroy(s);
    return PMF_ERR_OOM;
  }
  unsigned hw = std::thread::hardware_concurrency();
  s->pool.reset(new Pool(hw > 2 ? (int)std::min(hw - 1, 7u) : 0));
  *out = s;
  return PMF_OK;
}

int pmf_server_admit(pmf_server* s, const pmf_config* cfg, const pmf_meas* model, int* id_out) {
  if (!s || !cfg || !model || !id_out) return PMF_ERR_ARG;
  std::string why;
  int rc = validate_config(cfg, &why);
  if (rc) return sfail(s, rc, why);
  const int n = cfg->nx;
  if (cfg->transform == PMF_TRANSFORM_FFT && n != 1) {
    rc = PMF_ERR_UNSUPPORTED;
    why = "the FFT form exists in the 1-D kernel only";
  } else if (n == 1) {
    rc = tc1_supported(cfg, &why);
  } else {
    pmf_config c2 = *cfg;
    c2.precision = filter_precision(s, n);
    rc = tc_supported(&c2, &why);
  }
  if (rc) return sfail(s, rc, why);
  MeasParams mp;
  pmf_meas m = *model;
  for (int i = 0; i < PMF_MAX_NZ; ++i) m.z[i] = 0.0;
  rc = meas_params(n, &m, &mp, &why);
  if (rc) return sfail(s, rc, why);
  if (n == 2 && mp.nz > 2)   // the batched 2-D kernels form at most two likelihood components
    return sfail(s, PMF_ERR_UNSUPPORTED, "2-D filters take at most two measurement components");
  if (n == 3 && mp.kind == PMF_MEAS_RANGE)   // the 3-D pipelines: linear and bearing + linear
    return sfail(s, PMF_ERR_UNSUPPORTED, "3-D filters take linear and bearing + linear measurements");
  if (s->free_ids.empty()) return sfail(s, PMF_ERR_ADMISSION, "no free filter id");
  long long P = 1;
  for (int a = 0; a < n; ++a) P *= cfg->N[a];
  long long bytes = (long long)sizeof(DevState) + 8 * P + (long long)sizeof(MeasParams);
  if (n == 3) bytes += (long long)tc3_state_bytes();
  if (n == 2) bytes += (long long)tc_plan_bytes();
  // table kind of this filter's axes (the 2-D size-64 class has its own layout)
  int form2 = 0;
  if (n == 2) {
    pmf_config fc = *cfg;
    fc.precision = s->precision;
    form2 = tc2_form(&fc, s->s[0]);
  }
  const int cls = n == 2 ? tc_class_form(cfg->N[0], cfg->N[1], form2, s->precision) : 128;
  const int tkind = n == 1 ? 1 : (cls == 64 ? 3 : cls == 96 ? 4 : filter_precision(s, n) != s->precision ? 5 : 2);
  long long tbytes = 0;
  void* tab = nullptr;
  for (int a = 0; a < n; ++a) {
    bool seen = false;
    for (int b = 0; b < a; ++b) seen = seen || cfg->N[b] == cfg->N[a];
    if (!seen) table_for(s, tkind, cfg->N[a], &tab, nullptr, &tbytes, false);
  }
  if (s->budget && (size_t)(s->bytes + bytes + tbytes) > s->budget)
    return sfail(s, PMF_ERR_ADMISSION, "device-memory budget");

  const int id = s->free_ids.back();
  SFilter& f = s->f[id];
  f = SFilter{};
  f.cfg = *cfg;
  f.cfg.precision = filter_precision(s, n);
  f.cls = cls;
  f.mp = mp;
  f.P = P;
  bool ok = cudaMalloc(&f.st, sizeof(DevState)) == cudaSuccess &&
            cudaMalloc(&f.buf, sizeof(float) * 2 * P) == cudaSuccess &&
            cudaMalloc(&f.d_mp, sizeof(MeasParams)) == cudaSuccess;
  if (ok && n == 3) ok = tc3_alloc(&f.tc3) == PMF_OK;
  if (ok && n == 2) ok = cudaMalloc(&f.plan, tc_plan_bytes()) == cudaSuccess;
  size_t hb[3] = {0, 0, 0};
  void* tabs[3] = {nullptr, nullptr, nullptr};
  long long added = 0;
  for (int a = 0; a < n && ok; ++a) ok = table_for(s, tkind, cfg->N[a], &tabs[a], &hb[a], &added, true) == PMF_OK;
  s->bytes += added;
  if (!ok) {
    f.bytes = 0;
    free_filter(s, f);
    return sfail(s, PMF_ERR_OOM, "filter memory");
  }
  f.bytes = bytes;
  s->bytes += bytes;
  f.tct.prec = f.cfg.precision;
  for (int a = 0; a < n && n > 1; ++a) {
    f.tct.hart[a] = tabs[a];
    f.tct.hart_bytes[a] = hb[a];
  }
  // initial state and prior on the device (stream 0), then the slot entry
  DevState h = initial_state(f.cfg);
  double aux[kAuxSize] = {0};
  inv(n, cfg->P0, aux);
  for (int a = 0; a < n; ++a) aux[kAuxM0 + a] = cfg->m0[a];
  Dims d{};
  d.nx = n;
  d.P = P;
  for (int a = 0; a < MAXN; ++a) d.N[a] = a < n ? cfg->N[a] : 1;
  cudaStream_t st = s->s[0];
  ok = cudaMemcpyAsync(f.st, &h, sizeof(DevState), cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(f.d_mp, &mp, sizeof(MeasParams), cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(s->d_aux, aux, sizeof(aux), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok) s->launches += tc_prior(d, f.st, s->d_aux, f.buf, s->d_partials, st);
  if (ok && n == 1) {
    const Slot1 sl{f.st, f.buf, f.buf + P, (const float*)tabs[0], cfg->N[0], f.d_mp, nullptr,
                   tc1_form(cfg, tabs[0], st)};
    ok = cudaMemcpyAsync(s->d_slots1 + id, &sl, sizeof(sl), cudaMemcpyHostToDevice, st) == cudaSuccess;
  } else if (ok && n == 2) {
    FilterSlot sl{};
    sl.st = f.st;
    sl.buf0 = f.buf;
    sl.buf1 = f.buf + P;
    for (int a = 0; a < 2; ++a) {
      sl.hart[a] = (const uint8_t*)tabs[a];
      sl.sctab[a] = (const float*)((const uint8_t*)tabs[a] + hb[a]);
    }
    sl.N0 = cfg->N[0];
    sl.N1 = cfg->N[1];
    sl.mp = f.d_mp;
    sl.tc = nullptr;
    sl.plan = f.plan;
    sl.fft = form2;
    ok = cudaMemcpyAsync(s->d_slots2 + id, &sl, sizeof(sl), cudaMemcpyHostToDevice, st) == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess && cudaGetLastError() == cudaSuccess;
  if (!ok) {
    free_filter(s, f);
    return sfail(s, PMF_ERR_CUDA, "admission");
  }
  f.alive = true;
  s->free_ids.pop_back();
  *id_out = id;
  return PMF_OK;
}

int pmf_server_evict(pmf_server* s, int id) {
  if (!s || id < 0 || id >= s->cap || !s->f[id].alive) return PMF_ERR_ARG;
  if (s->f[id].busy || s->f[id].cur >= 0 || !s->f[id].queue.empty())
    return sfail(s, PMF_ERR_ARG, "filter has requests in progress");
  if (sync_all(s)) return sfail(s, PMF_ERR_CUDA, "synchronize");
  free_filter(s, s->f[id]);
  s->free_ids.push_back(id);
  return PMF_OK;
}

long long pmf_server_bytes(const pmf_server* s) { return s ? s->bytes : 0; }

int pmf_server_replay(pmf_server* s, long long n, const double* t_arrival, const int* ids, const double* z,
                      const double* taus, double* latency_out, double* stats_out) {
  if (!s || n < 0 || (n && (!t_arrival || !ids || !z || !taus))) return PMF_ERR_ARG;
  for (long long i = 0; i < n; ++i) {
    if (ids[i] < 0 || ids[i] >= s->cap || !s->f[ids[i]].alive) return sfail(s, PMF_ERR_ARG, "unknown filter id");
    if (!std::isfinite(taus[i]) || taus[i] < 0.0 || !std::isfinite(t_arrival[i]) ||
        (i && t_arrival[i] < t_arrival[i - 1]) || !finite_all(z + i * PMF_MAX_NZ, PMF_MAX_NZ))
      return sfail(s, PMF_ERR_ARG, "invalid request");
  }
  const long long l0 = s->launches, b0 = s->batches, i0 = s->items, m0 = s->max_batch;
  s->max_batch = 0;
  const double t0 = now_s();
  long long next = 0, done = 0;
  while (done < n) {
    const double t = now_s() - t0;
    while (next < n && t_arrival[next] <= t) {
      s->f[ids[next]].queue.push_back(next);
      mark_ready(s, ids[next]);
      ++next;
    }
    done += poll(s, t0, t_arrival, latency_out);
    if (!s->ready.empty() && s->inflight < kInflight) {
      const int rc = launch_batch(s, z, taus);
      if (rc) return rc;
    } else if (s->inflight == 0 && s->ready.empty() && next < n) {
      // idle until the next arrival
      const double wait = t_arrival[next] - (now_s() - t0);
      if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
    }
  }
  if (sync_all(s)) return sfail(s, PMF_ERR_CUDA, "synchronize");
  if (stats_out) {
    const double nb = (double)(s->batches - b0);
    stats_out[0] = now_s() - t0;
    stats_out[1] = nb;
    stats_out[2] = (double)(s->launches - l0);
    stats_out[3] = (double)s->max_batch;
    stats_out[4] = nb > 0 ? (double)(s->items - i0) / nb : 0.0;
    stats_out[5] = (double)n;
  }
  if (s->max_batch < m0) s->max_batch = m0;
  return PMF_OK;
}

int pmf_server_moments(pmf_server* s, int id, double* mean_out, double* cov_out) {
  if (!s || id < 0 || id >= s->cap || !s->f[id].alive) return PMF_ERR_ARG;
  if (sync_all(s)) return sfail(s, PMF_ERR_CUDA, "synchronize");
  SFilter& f = s->f[id];
  FrameState h;
  if (cudaMemcpy(&h, &f.st->f, sizeof(FrameState), cudaMemcpyDeviceToHost) != cudaSuccess)
    return sfail(s, PMF_ERR_CUDA, "copy");
  const int n = f.cfg.nx;
  if (mean_out) std::memcpy(mean_out, h.mean, sizeof(double) * n);
  if (cov_out) std::memcpy(cov_out, h.cov, sizeof(double) * n * n);
  if (h.status) {
    const int zero = 0;
    cudaMemcpy(&f.st->f.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return sfail(s, h.status, "device status");
  }
  return PMF_OK;
}

int pmf_server_get_pdf(pmf_server* s, int id, double* host_out, double* c_out, double* M_out) {
  if (!s || id < 0 || id >= s->cap || !s->f[id].alive) return PMF_ERR_ARG;
  if (sync_all(s)) return sfail(s, PMF_ERR_CUDA, "synchronize");
  SFilter& f = s->f[id];
  FrameState h;
  if (cudaMemcpy(&h, &f.st->f, sizeof(FrameState), cudaMemcpyDeviceToHost) != cudaSuccess)
    return sfail(s, PMF_ERR_CUDA, "copy");
  const int n = f.cfg.nx;
  if (c_out) std::memcpy(c_out, h.c, sizeof(double) * n);
  if (M_out) std::memcpy(M_out, h.M, sizeof(double) * n * n);
  if (host_out) {
    std::vector<float> tmp(f.P);
    if (cudaMemcpy(tmp.data(), f.buf + (h.cur ? f.P : 0), sizeof(float) * f.P, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return sfail(s, PMF_ERR_CUDA, "copy");
    for (long long i = 0; i < f.P; ++i) host_out[i] = h.pscale * (double)tmp[i];
  }
  return PMF_OK;
}

const char* pmf_server_last_error(const pmf_server* s) { return s ? s->err.c_str() : "null server"; }

void pmf_server_destroy(pmf_server* s) {
  if (!s) return;
  for (int k = 0; k < 3; ++k)
    if (s->s[k]) cudaStreamSynchronize(s->s[k]);
  for (auto& f : s->f)
    if (f.alive) free_filter(s, f);
  for (auto& kv : s->tables) cudaFree(kv.second);
  for (auto& b : s->ring) {
    for (int k = 0; k < 3; ++k)
      if (b.ev[k]) cudaEventDestroy(b.ev[k]);
    tc3_stage_free(&b.stage3);
    for (int k = 0; k < 2; ++k) {
      cudaFreeHost(b.h_items[k]);
      cudaFreeHost(b.h_tc[k]);
      cudaFree(b.d_items[k]);
      cudaFree(b.d_tc[k]);
    }
  }
  cudaFree(s->d_slots1);
  cudaFree(s->d_slots2);
  cudaFree(s->d_partials);
  cudaFree(s->d_aux);
  for (int k = 0; k < 3; ++k)
    if (s->s[k]) cudaStreamDestroy(s->s[k]);
  delete s;
}

}  // extern "C"
