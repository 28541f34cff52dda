// Runtime behind the C-ABI of include/sage.h: the per-GPU pool (the paper's
// unified memory daemon, Sec. 4.1), read-only sharing by key with reference
// counts (Sec. 6.2), staging of read-only data through a pinned ring on a side
// stream while the calling thread loads kernels and builds workspaces
// (parallelised setup, Sec. 5.1), the readiness gate before launch (Sec. 5.2),
// and the invocation chain of the recommendation-style function.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/mman.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/sage.h"
#include "kernels.h"

namespace sage {
static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

int device_sms() {
  static std::atomic<int> sms[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  int n = sms[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
  sms[dev].store(n, std::memory_order_relaxed);
  return n;
}
}  // namespace sage

using namespace sage;

namespace {

thread_local std::string t_err;

sage_status fail(sage_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}

}  // namespace

void sage::set_last_error(const char* msg) { t_err = msg; }

namespace {

#define SAGE_CK(call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return fail(SAGE_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------- pinned host memory
// Host memory the copy engines read fast: 2 MiB aligned, advised to transparent
// huge pages, then page-locked with cudaHostRegister.  (Small separate pinned
// allocations backed by 4 KiB pages copied at ~10 GB/s on the B300 hosts
// measured, slices of huge-page-backed memory at ~50 GB/s.)
constexpr size_t kHugePage = size_t(2) << 20;

void* host_alloc_pinned(size_t bytes, cudaError_t* err) {
  bytes = (bytes + kHugePage - 1) & ~(kHugePage - 1);
  void* p = nullptr;
  if (posix_memalign(&p, kHugePage, bytes) != 0 || !p) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  madvise(p, bytes, MADV_HUGEPAGE);
  *err = cudaHostRegister(p, bytes, cudaHostRegisterDefault);
  if (*err != cudaSuccess) {
    free(p);
    return nullptr;
  }
  return p;
}

void host_free_pinned(void* p) {
  if (!p) return;
  cudaHostUnregister(p);
  free(p);
}

// ---------------------------------------------------------------- host workers
// A fixed set of threads that run fn(i) for i in [0, n) together with the caller.
class Workers {
 public:
  explicit Workers(int n) {
    for (int i = 0; i < n; ++i) th_.emplace_back([this] { loop(); });
  }
  ~Workers() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void parallel_for(int n, const std::function<void(int)>& fn) {
    std::unique_lock<std::mutex> g(job_mu_);  // one job at a time
    {
      std::lock_guard<std::mutex> l(mu_);
      fn_ = &fn;
      n_ = n;
      next_ = 0;
      done_ = 0;
      ++gen_;
    }
    cv_.notify_all();
    run_items();
    std::unique_lock<std::mutex> l(mu_);
    done_cv_.wait(l, [&] { return done_ == n_; });
    fn_ = nullptr;
  }
  int size() const { return static_cast<int>(th_.size()) + 1; }

 private:
  void run_items() {
    for (;;) {
      int i;
      const std::function<void(int)>* f;
      {
        std::lock_guard<std::mutex> l(mu_);
        if (!fn_ || next_ >= n_) return;
        i = next_++;
        f = fn_;
      }
      (*f)(i);
      {
        std::lock_guard<std::mutex> l(mu_);
        if (++done_ == n_) done_cv_.notify_all();
      }
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> l(mu_);
        cv_.wait(l, [&] { return stop_ || (gen_ != seen && fn_ && next_ < n_); });
        if (stop_) return;
        seen = gen_;
      }
      run_items();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_, job_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0, next_ = 0, done_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

struct Layer {
  int in, out;
  const void* W;
  const float* b;
};

// One invocation slot: activations for `cap` rows and an I/O arena for host
// invocations; `done` orders the slot's reuse across streams.
struct Slot {
  int cap = 0;
  char* buf = nullptr;
  size_t bytes = 0;
  std::vector<char*> bot;  // bottom hidden outputs except the last layer's
  char* concat = nullptr;
  std::vector<char*> top;  // top hidden outputs except the head's
  // head fused into the last hidden layer: per-row group sums and arrival counters
  float* hpart = nullptr;
  unsigned* hcnt = nullptr;
  unsigned* gwork = nullptr;  // the gather's claimed-work counters {next, done}
  char* io = nullptr;
  size_t io_bytes = 0;
  cudaEvent_t done = nullptr;
  bool used = false;
  // the bottom MLP runs on `branch` beside the gather (fork / join events)
  cudaStream_t branch = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // host invocations: inputs are copied on `h2d` (after the slot's previous use)
  // so that they overlap the compute still running on the launch stream
  cudaStream_t h2d = nullptr;
  cudaEvent_t copied = nullptr;
  // CUDA graph of the launch chain: captured on `capture` for every batch, used to
  // update `exec` (same kernels, new parameters), which is launched in one call
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec = nullptr;
  // top hidden layers whose outputs the last launch chain wrote (the last hidden
  // layer is not written when the head runs in its epilogue)
  int top_written = 0;
  // false when the gather ran fused with the first top layer (no pooled columns written)
  bool pooled_written = true;
};

}  // namespace

struct sage_pool_s;

// Read-only data of one key kept in page-locked host memory (stage 2 of the
// multi-stage exit): the tables and weights items exactly as on the device.
struct HostImage {
  char* tables = nullptr;
  char* weights = nullptr;
  size_t tb = 0, wb = 0;
  std::string sig;     // shape signature the image belongs to
  uint64_t last = 0;   // LRU clock
  size_t bytes() const { return tb + wb; }
};

struct Entry {
  sage_pool_s* pool = nullptr;
  std::string key;
  int dtype = 0, T = 0, dim = 0, n_dense = 0;
  std::vector<int64_t> rows;
  std::vector<int> bot, top;
  size_t tables_bytes = 0, weights_bytes = 0, reserved = 0, ws_bytes = 0;
  char* d_tables = nullptr;
  char* d_weights = nullptr;
  int* d_err = nullptr;
  std::vector<Layer> layers;
  int64_t table_off[kMaxTables] = {};
  int refs = 0;
  std::string sig;        // shape signature (dtype, tables, layers, item sizes)
  // fp32 functions whose hidden layers all tile on the tensor cores keep every
  // activation as two planes (tf32 hi, fp32 residual lo) and the hidden-layer
  // weights split the same way (computed once after staging)
  bool presplit = false;
  char* d_wsplit = nullptr;
  size_t wsplit_bytes = 0;
  std::vector<std::pair<const float*, const float*>> wplanes;  // per layer: (hi, lo) or nulls
  HostImage owned;        // host image this entry was re-staged from (kept for the next demotion)
  // read-only items mapped from another process (cross-process sharing): no
  // staging here; a waiter thread opens the readiness gate when the owner reports
  // the data complete
  std::unique_ptr<sage::ImportedData> imp;
  std::thread imp_waiter;

  // staging (the read-only data's journey host -> device)
  sage_data_desc tdesc{}, wdesc{};
  std::mutex smu;
  std::condition_variable scv;
  int sstate = 0;      // 0 queued/copying, 1 all copies queued (ready event recorded), 2 failed
  int setup = 0;       // 0 building, 1 ready, 2 failed
  bool cancel = false;
  bool queued = false;
  cudaEvent_t ready = nullptr;
  Clock::time_point t_prepare;
  double stage_ms = 0, fill_ms = 0;
  int64_t staged_bytes = 0;

  // invocations
  std::mutex imu;
  std::vector<Slot> slots;
  int next_slot = 0;
  int max_batch = 4096;
  int last_slot = -1, last_M = 0;  // the slot and rows of the most recent batch

  int concat_dim() const { return T * dim + bot.back(); }
  size_t elem() const { return dtype == SAGE_BF16 ? 2 : 4; }
};

struct sage_fn_s {
  sage_pool_s* pool;
  Entry* e;
  uint64_t magic;
};
static constexpr uint64_t kFnMagic = 0x5A6E5F66756E6331ull;

struct sage_pool_s {
  int device = 0;
  size_t budget = 0, used = 0;
  sage_dev_alloc_fn dalloc = nullptr;
  sage_dev_free_fn dfree = nullptr;
  void* actx = nullptr;
  bool serial_setup = false;
  bool graphs = false;           // fused batches replayed through CUDA graphs
  bool exportable = false;       // read-only items in exportable VMM memory (shared with other processes)
  std::unordered_map<void*, sage::VmmBlock> vmm;  // exportable blocks by mapped address (under mu)
  cudaStream_t side = nullptr;   // staging copies
  cudaStream_t alloc = nullptr;  // allocations and frees (never waits behind staging copies)
  size_t chunk_bytes = 0;
  char* ring_mem = nullptr;  // one pinned, huge-page-backed allocation for all chunks
  std::vector<char*> ring;
  std::vector<cudaEvent_t> ring_ev;
  size_t ring_next = 0;
  std::unique_ptr<Workers> workers;
  std::thread stager;
  std::mutex qmu;
  std::condition_variable qcv;
  std::deque<Entry*> queue;
  bool stop = false;
  std::mutex mu;
  std::unordered_map<std::string, Entry*> entries;
  std::unordered_set<sage_fn_s*> handles;
  // stage-2 host cache of released keys' read-only data
  size_t host_budget = 0, host_used = 0;
  std::unordered_map<std::string, HostImage> hcache;
  uint64_t hclock = 0;
  sage_pool_stats_t st{};
  std::atomic<int64_t> h2d{0}, invocations{0};

  void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    if (dalloc) return dalloc(bytes, s, actx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void dev_free(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (dfree) dfree(p, bytes, s, actx);
    else cudaFreeAsync(p, s);
  }
  // Read-only items (tables, weights): exportable VMM blocks when the pool shares
  // them with other processes, otherwise ordinary device memory.
  void* ro_alloc(size_t bytes, cudaStream_t s) {
    if (!exportable) return dev_alloc(bytes, s);
    sage::VmmBlock b;
    if (!sage::vmm_alloc(device, bytes ? bytes : 256, &b)) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    vmm[b.va] = b;
    return b.va;
  }
  // Every use of p must have finished (VMM blocks are unmapped at once).
  void ro_free(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (!exportable) return dev_free(p, bytes, s);
    sage::VmmBlock b;
    {
      std::lock_guard<std::mutex> g(mu);
      auto it = vmm.find(p);
      if (it == vmm.end()) return;
      b = it->second;
      vmm.erase(it);
    }
    sage::vmm_free(b);
  }
};

namespace {

// ---------------------------------------------------------------- staging daemon

bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

std::string shape_sig(const sage_fn_desc* d) {
  std::string s = std::to_string(d->dtype) + "|" + std::to_string(d->num_tables) + "|" + std::to_string(d->dim) +
                  "|" + std::to_string(d->n_dense) + "|";
  for (int t = 0; t < d->num_tables; ++t) s += std::to_string(d->rows[t]) + ",";
  s += "|";
  for (int l = 0; l < d->n_bot; ++l) s += std::to_string(d->bot_dims[l]) + ",";
  s += "|";
  for (int l = 0; l < d->n_top; ++l) s += std::to_string(d->top_dims[l]) + ",";
  return s + "|" + std::to_string(d->tables.bytes) + "|" + std::to_string(d->weights.bytes);
}

void free_image(sage_pool_s* P, HostImage& h) {
  if (h.tables) host_free_pinned(h.tables);
  if (h.weights) host_free_pinned(h.weights);
  P->host_used -= std::min(P->host_used, h.bytes());
  h = HostImage();
}

// Make room for `need` bytes of host images (P->mu held); false if impossible.
bool host_cache_make_room(sage_pool_s* P, size_t need) {
  if (need > P->host_budget) return false;
  while (P->host_used + need > P->host_budget && !P->hcache.empty()) {
    auto victim = P->hcache.begin();
    for (auto it = P->hcache.begin(); it != P->hcache.end(); ++it)
      if (it->second.last < victim->second.last) victim = it;
    free_image(P, victim->second);
    P->hcache.erase(victim);
  }
  return P->host_used + need <= P->host_budget;
}

// Stage one data item into dst: fill pinned ring chunks on the host workers and
// copy each on the side stream; a chunk is refilled only after its previous
// copy finished.  Returns false if the producer failed or staging was cancelled.
bool stage_item(sage_pool_s* P, Entry* e, const sage_data_desc& d, char* dst, double* fill_ms) {
  if (d.bytes == 0) return true;
  if (d.host_src && is_pinned(d.host_src)) {
    if (cudaMemcpyAsync(dst, d.host_src, d.bytes, cudaMemcpyHostToDevice, P->side) != cudaSuccess) return false;
    P->h2d += static_cast<int64_t>(d.bytes);
    e->staged_bytes += static_cast<int64_t>(d.bytes);
    return true;
  }
  const int parts_per_chunk = P->workers->size();
  for (size_t off = 0; off < d.bytes; off += P->chunk_bytes) {
    {
      std::lock_guard<std::mutex> g(e->smu);
      if (e->cancel) return false;
    }
    const size_t n = std::min(P->chunk_bytes, d.bytes - off);
    const size_t k = P->ring_next++ % P->ring.size();
    if (cudaEventSynchronize(P->ring_ev[k]) != cudaSuccess) return false;
    char* buf = P->ring[k];
    std::atomic<int> bad{0};
    const size_t part = align256((n + parts_per_chunk - 1) / parts_per_chunk);
    const int nparts = static_cast<int>((n + part - 1) / part);
    auto t0 = Clock::now();
    P->workers->parallel_for(nparts, [&](int i) {
      const size_t p0 = static_cast<size_t>(i) * part;
      const size_t pn = std::min(part, n - p0);
      if (d.host_src) {
        memcpy(buf + p0, static_cast<const char*>(d.host_src) + off + p0, pn);
      } else if (d.fill(buf + p0, off + p0, pn, d.fill_ctx) != 0) {
        bad.store(1);
      }
    });
    *fill_ms += ms_since(t0);
    if (bad.load()) return false;
    if (cudaMemcpyAsync(dst + off, buf, n, cudaMemcpyHostToDevice, P->side) != cudaSuccess) return false;
    if (cudaEventRecord(P->ring_ev[k], P->side) != cudaSuccess) return false;
    P->h2d += static_cast<int64_t>(n);
    e->staged_bytes += static_cast<int64_t>(n);
  }
  return true;
}

// After the read-only items are in place (or failed): the split weight planes,
// the ready event and the entry's staging state.
void finish_staging(sage_pool_s* P, Entry* e, bool ok, double fill_ms) {
  if (ok && e->presplit) {
    for (size_t l = 0; l < e->wplanes.size(); ++l) {
      if (!e->wplanes[l].first) continue;
      const Layer& L = e->layers[l];
      if (launch_split_planes(static_cast<const float*>(L.W), const_cast<float*>(e->wplanes[l].first),
                              const_cast<float*>(e->wplanes[l].second), static_cast<size_t>(L.in) * L.out,
                              P->side) != cudaSuccess)
        ok = false;
    }
  }
  // the ready event covers every copy queued for this entry, also on failure
  if (cudaEventRecord(e->ready, P->side) != cudaSuccess) ok = false;
  const double stage_ms = ms_since(e->t_prepare);
  {
    std::lock_guard<std::mutex> g(P->mu);
    P->st.last_stage_ms = stage_ms;
    P->st.last_fill_ms = fill_ms;
  }
  std::lock_guard<std::mutex> g(e->smu);
  e->stage_ms = stage_ms;
  e->fill_ms = fill_ms;
  e->sstate = ok ? 1 : 2;
  e->scv.notify_all();
}

void stage_entry(sage_pool_s* P, Entry* e) {
  double fill_ms = 0;
  const bool ok = stage_item(P, e, e->wdesc, e->d_weights, &fill_ms) &&
                  stage_item(P, e, e->tdesc, e->d_tables, &fill_ms);
  finish_staging(P, e, ok, fill_ms);
}

void stager_loop(sage_pool_s* P) {
  cudaSetDevice(P->device);
  for (;;) {
    Entry* e;
    {
      std::unique_lock<std::mutex> l(P->qmu);
      P->qcv.wait(l, [&] { return P->stop || !P->queue.empty(); });
      if (P->queue.empty()) return;
      e = P->queue.front();
      P->queue.pop_front();
    }
    stage_entry(P, e);
  }
}

// ---------------------------------------------------------------- kernel timing

enum ProfKind {
  kProfBottom0 = 0,
  kProfGemmF32,
  kProfGemmTc,
  kProfGather,
  kProfHead,
  kProfGemmTf32,
  kProfBottom01,
  kProfGatherTop0,
  kProfKinds
};
const char* const kProfNames[kProfKinds] = {"bottom0", "gemm_f32",    "gemm_tc",  "gather",
                                            "head",    "gemm_tf32x3", "bottom01", "gather_top0"};

struct ProfRec {
  int kind;
  double work;
  cudaEvent_t a, b;
};

std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;

// Brackets one launch with timing events on its stream while profiling is on.
struct ProfScope {
  cudaStream_t s;
  int kind;
  double work;
  cudaEvent_t a = nullptr;
  ProfScope(cudaStream_t s_, int kind_, double work_) : s(s_), kind(kind_), work(work_) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    if (cudaEventCreate(&a) != cudaSuccess) {
      a = nullptr;
      return;
    }
    cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back({kind, work, a, b});
  }
};

// ---------------------------------------------------------------- kernels / workspace

std::once_flag g_load_once;
double g_load_ms = 0;

double load_kernels_once() {
  double spent = 0;
  std::call_once(g_load_once, [&] {
    auto t0 = Clock::now();
    preload_gather_kernels();
    preload_simt_kernels();
    preload_tc_kernels();
    preload_tf32_kernels();
    preload_bottom01_kernels();
    preload_gather_top0_kernels();
    g_load_ms = ms_since(t0);
    spent = g_load_ms;
  });
  return spent;
}

// planes per activation buffer: 2 (hi, lo) for pre-split fp32 functions
size_t planes(const Entry* e) { return e->presplit ? 2 : 1; }

// Groups of 64 columns of the last hidden top layer when the head can be fused
// into its epilogue (tensor-core layer, N / 64 a power of two), else 0.
int head_groups(const Entry* e) {
  if (e->top.size() < 2) return 0;
  const int N = e->top[e->top.size() - 2];
  const int G = N / 64;
  if (N % 64 || G < 1 || (G & (G - 1))) return 0;
  return (e->dtype == SAGE_BF16 || e->presplit) ? G : 0;
}

size_t slot_bytes(const Entry* e, int cap) {
  size_t b = 0;
  const size_t pl = planes(e);
  for (size_t l = 0; l + 1 < e->bot.size(); ++l)
    b += align256(pl * static_cast<size_t>(cap) * e->bot[l] * e->elem());
  b += align256(pl * static_cast<size_t>(cap) * e->concat_dim() * e->elem());
  for (size_t l = 0; l + 1 < e->top.size(); ++l)
    b += align256(pl * static_cast<size_t>(cap) * e->top[l] * e->elem());
  if (const int G = head_groups(e)) b += align256(static_cast<size_t>(cap) * G * 4) + align256(static_cast<size_t>(cap) * 4);
  b += align256(2 * sizeof(unsigned));
  return b;
}

sage_status build_slot(Entry* e, Slot& s, int cap, cudaStream_t stream) {
  sage_pool_s* P = e->pool;
  const size_t bytes = slot_bytes(e, cap);
  char* buf = static_cast<char*>(P->dev_alloc(bytes, stream));
  if (!buf) return fail(SAGE_ERR_NOMEM, "workspace allocation of %zu bytes failed", bytes);
  if (s.buf) P->dev_free(s.buf, s.bytes, stream);
  s.buf = buf;
  s.bytes = bytes;
  s.cap = cap;
  s.bot.clear();
  s.top.clear();
  size_t o = 0;
  const size_t pl = planes(e);
  for (size_t l = 0; l + 1 < e->bot.size(); ++l) {
    s.bot.push_back(buf + o);
    o += align256(pl * static_cast<size_t>(cap) * e->bot[l] * e->elem());
  }
  s.concat = buf + o;
  o += align256(pl * static_cast<size_t>(cap) * e->concat_dim() * e->elem());
  for (size_t l = 0; l + 1 < e->top.size(); ++l) {
    s.top.push_back(buf + o);
    o += align256(pl * static_cast<size_t>(cap) * e->top[l] * e->elem());
  }
  s.hpart = nullptr;
  s.hcnt = nullptr;
  if (const int G = head_groups(e)) {
    s.hpart = reinterpret_cast<float*>(buf + o);
    o += align256(static_cast<size_t>(cap) * G * 4);
    s.hcnt = reinterpret_cast<unsigned*>(buf + o);
    o += align256(static_cast<size_t>(cap) * 4);
    SAGE_CK(cudaMemsetAsync(s.hcnt, 0, static_cast<size_t>(cap) * 4, stream));
  }
  s.gwork = reinterpret_cast<unsigned*>(buf + o);
  o += align256(2 * sizeof(unsigned));
  SAGE_CK(cudaMemsetAsync(s.gwork, 0, 2 * sizeof(unsigned), stream));
  return SAGE_OK;
}

sage_status check_shape_impl(const sage_fn_desc* d) {
  if (!d || !d->fn_key) return fail(SAGE_ERR_INVALID, "null descriptor or key");
  if (strlen(d->fn_key) == 0 || strlen(d->fn_key) > 200) return fail(SAGE_ERR_INVALID, "key length must be 1..200");
  if (d->dtype != SAGE_F32 && d->dtype != SAGE_BF16) return fail(SAGE_ERR_INVALID, "bad dtype");
  if (d->num_tables < 1 || d->num_tables > kMaxTables || !d->rows) return fail(SAGE_ERR_INVALID, "bad num_tables");
  const int es = d->dtype == SAGE_BF16 ? 2 : 4;
  const int rb = d->dim * es;
  if (d->dim < 1 || rb < 16 || rb > 1024 || (rb & (rb - 1)))
    return fail(SAGE_ERR_INVALID, "dim*elem must be a power of two in [16, 1024] bytes");
  if (d->n_dense < 1 || d->n_dense > 64) return fail(SAGE_ERR_INVALID, "n_dense must be in [1, 64]");
  if (d->n_bot < 1 || d->n_bot > 8 || d->n_top < 1 || d->n_top > 8 || !d->bot_dims || !d->top_dims)
    return fail(SAGE_ERR_INVALID, "n_bot/n_top must be in [1, 8]");
  if (d->top_dims[d->n_top - 1] != 1) return fail(SAGE_ERR_INVALID, "the last top layer must have 1 output");
  size_t tb = 0;
  for (int t = 0; t < d->num_tables; ++t) {
    if (d->rows[t] < 1 || d->rows[t] >= (int64_t(1) << 31)) return fail(SAGE_ERR_INVALID, "bad rows[%d]", t);
    tb += static_cast<size_t>(d->rows[t]) * d->dim * es;
  }
  if (d->tables.bytes != tb) return fail(SAGE_ERR_INVALID, "tables.bytes %zu != %zu", d->tables.bytes, tb);
  if (d->tables.access != SAGE_READONLY || d->weights.access != SAGE_READONLY)
    return fail(SAGE_ERR_INVALID, "tables and weights must be SAGE_READONLY");
  // layer shapes
  std::vector<std::pair<int, int>> L;
  int prev = d->n_dense;
  for (int l = 0; l < d->n_bot; ++l) {
    if (d->bot_dims[l] < 1) return fail(SAGE_ERR_INVALID, "bad bot_dims");
    L.push_back({prev, d->bot_dims[l]});
    prev = d->bot_dims[l];
  }
  prev = d->num_tables * d->dim + d->bot_dims[d->n_bot - 1];
  for (int l = 0; l < d->n_top; ++l) {
    if (d->top_dims[l] < 1) return fail(SAGE_ERR_INVALID, "bad top_dims");
    L.push_back({prev, d->top_dims[l]});
    prev = d->top_dims[l];
  }
  size_t wb = 0;
  for (auto& p : L) {
    wb = align256(wb) + static_cast<size_t>(p.first) * p.second * es;
    wb = align256(wb) + static_cast<size_t>(p.second) * 4;
  }
  wb = align256(wb);
  if (d->weights.bytes != wb) return fail(SAGE_ERR_INVALID, "weights.bytes %zu != %zu", d->weights.bytes, wb);
  for (size_t l = 1; l + 1 < L.size(); ++l) {
    const int K = L[l].first, N = L[l].second;
    if (d->dtype == SAGE_BF16 && ((K % 64) || (N % 64)))
      return fail(SAGE_ERR_INVALID, "bf16 layer %zu (%d -> %d) needs multiples of 64", l, K, N);
    if (d->dtype == SAGE_F32 && ((K % 4) || (N % 4)))
      return fail(SAGE_ERR_INVALID, "fp32 layer %zu (%d -> %d) needs multiples of 4", l, K, N);
  }
  if (d->dtype == SAGE_BF16 && d->n_bot == 1 && ((d->num_tables * d->dim) % 8))
    return fail(SAGE_ERR_INVALID, "bad concat alignment");
  if (d->max_batch < 0 || d->workspace_slots < 0 || d->workspace_slots > 64)
    return fail(SAGE_ERR_INVALID, "bad max_batch/workspace_slots");
  return SAGE_OK;
}

sage_status check_desc(const sage_fn_desc* d) {
  sage_status st = check_shape_impl(d);
  if (st != SAGE_OK) return st;
  if ((!d->tables.host_src) == (!d->tables.fill) || (!d->weights.host_src) == (!d->weights.fill))
    return fail(SAGE_ERR_INVALID, "each data item needs exactly one of host_src or fill");
  return SAGE_OK;
}

bool same_shape(const Entry* e, const sage_fn_desc* d) {
  if (e->dtype != d->dtype || e->T != d->num_tables || e->dim != d->dim || e->n_dense != d->n_dense) return false;
  if (static_cast<int>(e->bot.size()) != d->n_bot || static_cast<int>(e->top.size()) != d->n_top) return false;
  for (int t = 0; t < e->T; ++t)
    if (e->rows[t] != d->rows[t]) return false;
  for (int l = 0; l < d->n_bot; ++l)
    if (e->bot[l] != d->bot_dims[l]) return false;
  for (int l = 0; l < d->n_top; ++l)
    if (e->top[l] != d->top_dims[l]) return false;
  return e->tables_bytes == d->tables.bytes && e->weights_bytes == d->weights.bytes;
}

// Free an entry's device memory after all of its work finished.  Returns the first
// error the waits for that work reported (a kernel or copy of the function that
// failed after its caller last checked); the memory is freed either way.
cudaError_t destroy_entry(sage_pool_s* P, Entry* e) {
  cudaError_t first = cudaSuccess;
  auto note = [&](cudaError_t c) {
    if (c != cudaSuccess && first == cudaSuccess) first = c;
  };
  if (e->imp) e->imp->interrupt();  // a waiter still blocked on the owner returns (failed)
  {
    std::unique_lock<std::mutex> l(e->smu);
    e->cancel = true;
    e->scv.wait(l, [&] { return e->sstate != 0; });
  }
  if (e->imp_waiter.joinable()) e->imp_waiter.join();
  if (e->ready) note(cudaEventSynchronize(e->ready));
  for (auto& s : e->slots) {
    if (s.done) {
      note(cudaEventSynchronize(s.done));
      cudaEventDestroy(s.done);
    }
    if (s.branch) {
      note(cudaStreamSynchronize(s.branch));
      cudaStreamDestroy(s.branch);
    }
    if (s.fork) cudaEventDestroy(s.fork);
    if (s.join) cudaEventDestroy(s.join);
    if (s.h2d) {
      note(cudaStreamSynchronize(s.h2d));
      cudaStreamDestroy(s.h2d);
    }
    if (s.copied) cudaEventDestroy(s.copied);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.capture) cudaStreamDestroy(s.capture);
  }
  // stage 2 of the multi-stage exit: keep the read-only data in the host cache
  bool ok_data = false;
  {
    std::lock_guard<std::mutex> g(e->smu);
    ok_data = e->sstate == 1 && e->setup == 1 && !e->imp;  // imported data is the owner's to keep
  }
  if (P->host_budget > 0 && ok_data) {
    std::unique_lock<std::mutex> g(P->mu);
    HostImage img = e->owned;
    e->owned = HostImage();
    bool have = img.tables != nullptr;
    if (!have && host_cache_make_room(P, e->tables_bytes + e->weights_bytes)) {
      cudaError_t he = cudaSuccess;
      img.tables = static_cast<char*>(host_alloc_pinned(e->tables_bytes, &he));
      img.weights = static_cast<char*>(host_alloc_pinned(e->weights_bytes, &he));
      img.tb = e->tables_bytes;
      img.wb = e->weights_bytes;
      if (img.tables && img.weights) {
        P->host_used += img.bytes();
        g.unlock();
        bool copied = cudaMemcpyAsync(img.tables, e->d_tables, img.tb, cudaMemcpyDeviceToHost, P->alloc) ==
                          cudaSuccess &&
                      cudaMemcpyAsync(img.weights, e->d_weights, img.wb, cudaMemcpyDeviceToHost, P->alloc) ==
                          cudaSuccess &&
                      cudaStreamSynchronize(P->alloc) == cudaSuccess;
        g.lock();
        have = copied;
        if (!copied) free_image(P, img);
      } else {
        if (img.tables) host_free_pinned(img.tables);
        if (img.weights) host_free_pinned(img.weights);
        img = HostImage();
      }
    }
    if (have) {
      img.sig = e->sig;
      img.last = ++P->hclock;
      auto old = P->hcache.find(e->key);
      if (old != P->hcache.end()) {
        free_image(P, old->second);
        P->hcache.erase(old);
      }
      P->hcache[e->key] = img;
      P->st.demotions++;
    }
  } else if (e->owned.tables) {
    std::lock_guard<std::mutex> g(P->mu);
    free_image(P, e->owned);
  }
  // every use of the entry's memory has finished (ready + slot events above)
  for (auto& s : e->slots) {
    P->dev_free(s.buf, s.bytes, P->alloc);
    P->dev_free(s.io, s.io_bytes, P->alloc);
  }
  if (!e->imp) {
    P->ro_free(e->d_tables, e->tables_bytes, P->alloc);
    P->ro_free(e->d_weights, e->weights_bytes, P->alloc);
  }
  P->dev_free(e->d_wsplit, e->wsplit_bytes, P->alloc);
  P->dev_free(e->d_err, 256, P->alloc);
  note(cudaStreamSynchronize(P->alloc));
  e->imp.reset();  // unmap the owner's copy after the last use above
  if (e->ready) cudaEventDestroy(e->ready);
  {
    std::lock_guard<std::mutex> g(P->mu);
    P->used -= e->reserved;
  }
  delete e;
  return first;
}

// Wait (host) until the entry's setup finished and all staging copies are queued.
sage_status wait_ready_enqueued(Entry* e) {
  std::unique_lock<std::mutex> l(e->smu);
  e->scv.wait(l, [&] { return e->sstate != 0 && e->setup != 0; });
  if (e->sstate == 2) return fail(SAGE_ERR_STAGING, "staging of '%s' failed", e->key.c_str());
  if (e->setup == 2) return fail(SAGE_ERR_CUDA, "setup of '%s' failed", e->key.c_str());
  return SAGE_OK;
}

bool valid_fn(sage_fn f) { return f && f->magic == kFnMagic && f->e; }

// fp32 dense layer: tensor cores (3 x tf32) when the shape tiles (N multiple of 64,
// 16-byte rows), otherwise the CUDA-core kernel.
bool f32_on_tensor_cores(int N, int K, int ldx, int ldy) { return N % 64 == 0 && K % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0; }

cudaError_t launch_f32_layer(int M, int N, int K, const float* x, int ldx, const float* W, const float* b, int relu,
                             float* y, int ldy, int* err, cudaStream_t s) {
  if (f32_on_tensor_cores(N, K, ldx, ldy))
    return launch_linear_f32_tc(M, N, K, x, ldx, W, b, relu, y, ldy, err, s, tuned_gemm(kGemmTf32x3, M, N, K));
  return launch_linear_f32(M, N, K, x, ldx, W, b, relu, y, ldy, s);
}

int f32_kind(int N, int K, int ldx, int ldy) {
  return f32_on_tensor_cores(N, K, ldx, ldy) ? kProfGemmTf32 : kProfGemmF32;
}

sage_status launch_chain(Entry* e, Slot& s, const InvTable& tab, cudaStream_t stream, bool confined = false) {
  const int M = tab.M;
  const int nb = static_cast<int>(e->bot.size()), nt = static_cast<int>(e->top.size());
  const size_t es = e->elem();
  const int cd = e->concat_dim();
  char* bot_out = s.concat + static_cast<size_t>(e->T) * e->dim * es;
  // pre-split fp32: the lo plane of a buffer with row stride ld sits cap*ld floats after its hi plane
  const bool ps2 = e->presplit;
  auto lo_of = [&](const void* hi, int ld) -> float* {
    return ps2 ? const_cast<float*>(static_cast<const float*>(hi)) + static_cast<size_t>(s.cap) * ld : nullptr;
  };
  auto f32_presplit = [&](const Layer& L, int l, const void* x, int ldx, void* y, int ldy) -> cudaError_t {
    return launch_linear_f32_tc_presplit(M, L.out, L.in, static_cast<const float*>(x), lo_of(x, ldx), ldx,
                                         e->wplanes[l].first, e->wplanes[l].second, L.b, 1,
                                         static_cast<float*>(y), lo_of(y, ldy), ldy, e->d_err, stream,
                                         tuned_gemm(kGemmTf32Pre, M, L.out, L.in));
  };
  // fork: the bottom MLP (columns [T*dim, cd) of the concat buffer) runs on the
  // slot's branch stream while the gather (columns [0, T*dim)) runs on `stream`
  // (while kernel timing is on, the branch is serialised so that each kernel's
  // events measure it alone; on a confined stream -- an SM partition -- it stays
  // on that stream so that every kernel runs on the partition's SMs)
  // the gather and the first top layer as one kernel (pre-split fp32 functions with
  // 64-column tables), when tuning kind 5 asks for it ((256, 2); untuned or (1, 1):
  // separate kernels, which measured faster on the batching workload -- the fused
  // kernel's one CTA per SM keeps half the gather's loads in flight).  It reads the
  // bottom MLP's output, so the bottom MLP then runs first, on the launch stream.
  bool fuse_g0 = false;
  if (ps2 && nt >= 2 && gather_top0_fusable(e->dtype, e->dim, e->T, e->bot.back(), e->top[0], true)) {
    const GemmCfg c = tuned_gemm(kGatherTop0, M, e->top[0], cd);
    fuse_g0 = c.bn == 256;
  }
  const bool overlap = !g_prof_on.load(std::memory_order_relaxed) && !confined && !fuse_g0;
  SAGE_CK(cudaEventRecord(s.fork, stream));
  SAGE_CK(cudaStreamWaitEvent(s.branch, s.fork, 0));
  const cudaStream_t main_stream = stream;
  if (overlap) stream = s.branch;
  // bottom MLP (layer 0 reads each invocation's dense rows); on the pre-split fp32
  // path layers 0 and 1 run as one kernel unless the tuning table says otherwise
  // (and layer 2 too, when the shape allows one whole-row tile per SM)
  int l1 = 1;
  if (ps2 && nb >= 2 && bottom01_fusable(e->layers[0].in, e->layers[0].out, e->layers[1].out)) {
    const Layer& L0 = e->layers[0];
    const Layer& L1 = e->layers[1];
    GemmCfg c = tuned_gemm(kBottom01, M, L1.out, L1.in);
    // untuned: a persistent CTA spends ~30 us on its tile whatever M is, so below
    // about 64 tiles the separate kernels, spread over more CTAs, finish first
    if (c.bn == 0 && (M + 127) / 128 < 64) c = GemmCfg{1, 1};
    if (c.bn != 1) {
      const bool three = nb >= 3 && (c.bn == 0 || c.stages == 202) &&
                         bottom012_fusable(L1.out, e->layers[2].out, M);
      const int last = three ? 2 : 1;
      void* y = last == nb - 1 ? bot_out : s.bot[last];
      const int ldy = last == nb - 1 ? cd : e->bot[last];
      double flops = 2.0 * M * (L0.in * L0.out + L1.in * L1.out);
      if (three) flops += 2.0 * M * e->layers[2].in * e->layers[2].out;
      ProfScope ps(stream, kProfBottom01, flops);
      int done = 0;
      SAGE_CK(launch_bottom01_f32(tab, L0.in, L0.out, static_cast<const float*>(L0.W), L0.b, L1.out,
                                  e->wplanes[1].first, e->wplanes[1].second, L1.b, static_cast<float*>(y),
                                  lo_of(y, ldy), ldy, e->d_err, stream, three ? GemmCfg{256, 202} : c,
                                  three ? e->wplanes[2].first : nullptr, three ? e->wplanes[2].second : nullptr,
                                  three ? e->layers[2].b : nullptr, three ? e->layers[2].out : 0, &done));
      if (done != last + 1) return fail(SAGE_ERR_CUDA, "fused bottom kernel ran %d layers, expected %d", done, last + 1);
      l1 = last + 1;
    }
  }
  if (l1 == 1) {
    const Layer& L0 = e->layers[0];
    void* y = nb == 1 ? bot_out : s.bot[0];
    const int ldy = nb == 1 ? cd : e->bot[0];
    ProfScope ps(stream, kProfBottom0, 2.0 * M * L0.in * L0.out);
    SAGE_CK(launch_bottom0(e->dtype, tab, L0.in, L0.out, L0.W, L0.b, y, ldy, stream, lo_of(y, ldy)));
  }
  for (int l = l1; l < nb; ++l) {
    const Layer& L = e->layers[l];
    const void* x = s.bot[l - 1];
    void* y = l == nb - 1 ? bot_out : s.bot[l];
    const int ldy = l == nb - 1 ? cd : e->bot[l];
    ProfScope ps(stream, e->dtype == SAGE_BF16 ? kProfGemmTc : f32_kind(L.out, L.in, L.in, ldy),
                 2.0 * M * L.in * L.out);
    if (e->dtype == SAGE_BF16)
      SAGE_CK(launch_linear_bf16_tc(M, L.out, L.in, x, L.in, L.W, L.b, 1, y, ldy, e->d_err, stream,
                                    tuned_gemm(kGemmBf16, M, L.out, L.in)));
    else if (ps2)
      SAGE_CK(f32_presplit(L, l, x, L.in, y, ldy));
    else
      SAGE_CK(launch_f32_layer(M, L.out, L.in, static_cast<const float*>(x), L.in, static_cast<const float*>(L.W),
                               L.b, 1, static_cast<float*>(y), ldy, e->d_err, stream));
  }
  SAGE_CK(cudaEventRecord(s.join, overlap ? s.branch : main_stream));
  stream = main_stream;
  // embedding-bag gather into the concat columns [0, T*dim)
  {
    GatherArgs a;
    a.dtype = e->dtype;
    a.tables = e->d_tables;
    for (int t = 0; t < e->T; ++t) {
      a.table_off[t] = e->table_off[t];
      a.table_rows[t] = static_cast<int32_t>(e->rows[t]);
    }
    a.T = e->T;
    a.dim = e->dim;
    a.out = s.concat;
    a.ldo = cd;
    a.err = e->d_err;
    a.out_lo = lo_of(s.concat, cd);
    a.work = s.gwork;
    // algorithmic bytes: each lookup reads a row and its index, each bag reads its
    // offset and writes one pooled row
    double lookups = 0;
    for (int i = 0; i < tab.n; ++i) lookups += static_cast<double>(tab.d[i].nidx);
    const double row = static_cast<double>(e->dim) * es;
    const double bytes = lookups * (row + 4.0) + static_cast<double>(e->T) * M * (8.0 + row);
    if (!fuse_g0) {
      ProfScope ps(stream, kProfGather, bytes);
      SAGE_CK(launch_gather(a, tab, stream));
    } else {
      // the bottom MLP ran on this stream already; the pooled columns stay on chip
      // (the work recorded is the gather's bytes without the pooled write)
      SAGE_CK(cudaStreamWaitEvent(stream, s.join, 0));
      const Layer& L = e->layers[nb];
      ProfScope ps(stream, kProfGatherTop0, bytes - static_cast<double>(e->T) * M * row);
      SAGE_CK(launch_gather_top0_f32(a, tab, L.out, L.in, reinterpret_cast<const float*>(s.concat),
                                     lo_of(s.concat, cd), cd, e->wplanes[nb].first, e->wplanes[nb].second, L.b,
                                     reinterpret_cast<float*>(s.top[0]), lo_of(s.top[0], L.out), L.out, e->d_err,
                                     stream));
    }
  }
  // join: the top MLP needs both halves of the concat buffer
  SAGE_CK(cudaStreamWaitEvent(stream, s.join, 0));
  // top MLP hidden layers (the first one is done when the gather ran fused with it)
  const int l0 = fuse_g0 ? 1 : 0;
  const char* x = fuse_g0 ? s.top[0] : s.concat;
  int ldx = fuse_g0 ? e->top[0] : cd;
  const Layer& H = e->layers[nb + nt - 1];
  s.top_written = l0;
  s.pooled_written = !fuse_g0;
  for (int l = l0; l + 1 < nt; ++l) {
    const Layer& L = e->layers[nb + l];
    char* y = s.top[l];
    if (l + 2 == nt && s.hcnt) {
      // the last hidden layer with the sigmoid head in its epilogue (when its tuned
      // tile configuration is a persistent one)
      const int kind = e->dtype == SAGE_BF16 ? kGemmBf16 : kGemmTf32Pre;
      GemmCfg c = tuned_gemm(kind, M, L.out, L.in);
      if (head_fusable(c, L.out) && c.bn < L.out) {
        // a persistent tile as wide as the layer finishes each row in registers
        GemmCfg cands[16];
        const int nc = gemm_candidates(kind, cands, 16);
        for (int i = 0; i < nc; ++i)
          if (cands[i].stages >= 100 && cands[i].bn == L.out) c = cands[i];
      }
      if (head_fusable(c, L.out)) {
        HeadParams hp;
        hp.f.w = H.W;
        hp.f.c = H.b;
        hp.f.part = s.hpart;
        hp.f.cnt = s.hcnt;
        hp.tab = tab;
        ProfScope ps(stream, e->dtype == SAGE_BF16 ? kProfGemmTc : kProfGemmTf32,
                     2.0 * M * L.in * L.out + 2.0 * M * H.in);
        if (e->dtype == SAGE_BF16)
          SAGE_CK(launch_linear_bf16_tc_head(M, L.out, L.in, x, ldx, L.W, L.b, 1, e->d_err, stream, c, hp));
        else
          SAGE_CK(launch_linear_f32_tc_presplit_head(M, L.out, L.in, reinterpret_cast<const float*>(x),
                                                     lo_of(x, ldx), ldx, e->wplanes[nb + l].first,
                                                     e->wplanes[nb + l].second, L.b, 1, e->d_err, stream, c, hp));
        return SAGE_OK;
      }
    }
    ProfScope ps(stream, e->dtype == SAGE_BF16 ? kProfGemmTc : f32_kind(L.out, L.in, ldx, L.out),
                 2.0 * M * L.in * L.out);
    if (e->dtype == SAGE_BF16)
      SAGE_CK(launch_linear_bf16_tc(M, L.out, L.in, x, ldx, L.W, L.b, 1, y, L.out, e->d_err, stream,
                                    tuned_gemm(kGemmBf16, M, L.out, L.in)));
    else if (ps2)
      SAGE_CK(f32_presplit(L, nb + l, x, ldx, y, L.out));
    else
      SAGE_CK(launch_f32_layer(M, L.out, L.in, reinterpret_cast<const float*>(x), ldx,
                               static_cast<const float*>(L.W), L.b, 1, reinterpret_cast<float*>(y), L.out,
                               e->d_err, stream));
    s.top_written = l + 1;
    x = y;
    ldx = L.out;
  }
  // sigmoid head, written to each invocation's out
  ProfScope ps(stream, kProfHead, 2.0 * M * H.in);
  SAGE_CK(launch_head(e->dtype, tab, H.in, x, ldx, H.W, H.b, stream, lo_of(x, ldx)));
  return SAGE_OK;
}

// Pick a slot able to hold M rows; called with e->imu held.
sage_status acquire_slot(Entry* e, int M, cudaStream_t stream, Slot** out, int which = -1) {
  if (which >= static_cast<int>(e->slots.size())) return fail(SAGE_ERR_INVALID, "slot %d out of range", which);
  Slot& s = which >= 0 ? e->slots[which] : e->slots[e->next_slot];
  if (which < 0) e->next_slot = (e->next_slot + 1) % static_cast<int>(e->slots.size());
  if (s.used) SAGE_CK(cudaStreamWaitEvent(stream, s.done, 0));
  if (M > s.cap) {
    // grow: wait for the slot's last use, then reallocate (rare)
    if (s.used) SAGE_CK(cudaEventSynchronize(s.done));
    int cap = std::max(M, s.cap + s.cap / 2);
    const size_t old_bytes = s.bytes;
    const size_t need = slot_bytes(e, cap);
    {
      std::lock_guard<std::mutex> g(e->pool->mu);
      if (need > old_bytes && e->pool->used + (need - old_bytes) > e->pool->budget)
        return fail(SAGE_ERR_NOMEM, "workspace growth to %d rows exceeds the pool budget", cap);
      if (need > old_bytes) {
        e->pool->used += need - old_bytes;
        e->reserved += need - old_bytes;
      }
    }
    sage_status st = build_slot(e, s, cap, stream);
    if (st != SAGE_OK) return st;
  }
  e->last_slot = static_cast<int>(&s - e->slots.data());
  e->last_M = M;
  *out = &s;
  return SAGE_OK;
}

// Capture the launch chain of one batch into the slot's graph executable (update
// in place when the kernels are the same as last time, else re-instantiate).
sage_status capture_chain(Entry* e, Slot& s, const InvTable& tab) {
  SAGE_CK(cudaStreamBeginCapture(s.capture, cudaStreamCaptureModeThreadLocal));
  sage_status st = launch_chain(e, s, tab, s.capture);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s.capture, &graph);
  if (st != SAGE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return fail(SAGE_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  bool updated = false;
  if (s.exec) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(s.exec, graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(s.exec);
      s.exec = nullptr;
    }
  }
  if (!updated) ce = cudaGraphInstantiate(&s.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    s.exec = nullptr;
    return fail(SAGE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  }
  return SAGE_OK;
}

sage_status run_batch(Entry* e, const InvTable& tab, cudaStream_t stream) {
  std::lock_guard<std::mutex> g(e->imu);
  Slot* s = nullptr;
  sage_status st = acquire_slot(e, tab.M, stream, &s);
  if (st != SAGE_OK) return st;
  SAGE_CK(cudaStreamWaitEvent(stream, e->ready, 0));
  const bool confined = sage::stream_is_confined(stream);
  if (e->pool->graphs && !confined && !g_prof_on.load(std::memory_order_relaxed)) {
    st = capture_chain(e, *s, tab);
    if (st != SAGE_OK) return st;
    SAGE_CK(cudaGraphLaunch(s->exec, stream));
  } else {
    st = launch_chain(e, *s, tab, stream, confined);
    if (st != SAGE_OK) return st;
  }
  SAGE_CK(cudaEventRecord(s->done, stream));
  s->used = true;
  return SAGE_OK;
}

}  // namespace

// ====================================================================== C-ABI

extern "C" {

const char* sage_last_error(void) { return t_err.c_str(); }

sage_status sage_host_alloc(size_t bytes, void** out) {
  if (!out || bytes == 0) return fail(SAGE_ERR_INVALID, "bad host allocation request");
  cudaError_t e = cudaSuccess;
  *out = host_alloc_pinned(bytes, &e);
  if (!*out) return fail(SAGE_ERR_NOMEM, "pinned host allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
  return SAGE_OK;
}

sage_status sage_host_free(void* p) {
  host_free_pinned(p);
  return SAGE_OK;
}

int64_t sage_kernel_launches(void) { return sage::launches(); }

sage_status sage_profile_enable(int on) {
  g_prof_on.store(on != 0);
  return SAGE_OK;
}

int sage_profile_read(sage_kernel_time* out, int max) {
  if (!out || max < 0) return fail(SAGE_ERR_INVALID, "bad output");
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    recs.swap(g_prof);
  }
  sage_kernel_time agg[kProfKinds];
  memset(agg, 0, sizeof(agg));
  sage_status st = SAGE_OK;
  for (auto& r : recs) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      st = fail(SAGE_ERR_CUDA, "profile events");
    agg[r.kind].launches++;
    agg[r.kind].total_ms += ms;
    agg[r.kind].work += r.work;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (st != SAGE_OK) return st;
  int n = 0;
  for (int k = 0; k < kProfKinds && n < max; ++k) {
    if (!agg[k].launches) continue;
    out[n] = agg[k];
    snprintf(out[n].name, sizeof(out[n].name), "%s", kProfNames[k]);
    ++n;
  }
  return n;
}

sage_status sage_pool_create(const sage_pool_config* cfg, sage_pool* out) {
  if (!out) return fail(SAGE_ERR_INVALID, "null out");
  *out = nullptr;
  sage_pool_config c{};
  if (cfg) c = *cfg;
  if ((c.dev_alloc == nullptr) != (c.dev_free == nullptr))
    return fail(SAGE_ERR_INVALID, "set both dev_alloc and dev_free or neither");
  auto t0 = Clock::now();
  SAGE_CK(cudaSetDevice(c.device));
  SAGE_CK(cudaFree(nullptr));  // create / bind the context
  std::unique_ptr<sage_pool_s> P(new sage_pool_s());
  P->device = c.device;
  P->dalloc = c.dev_alloc;
  P->dfree = c.dev_free;
  P->actx = c.alloc_ctx;
  P->serial_setup = c.serial_setup != 0;
  P->host_budget = c.host_cache_bytes;
  P->graphs = c.graphs != 0;
  P->exportable = c.exportable != 0;
  size_t free_b = 0, total_b = 0;
  SAGE_CK(cudaMemGetInfo(&free_b, &total_b));
  const size_t margin = size_t(2) << 30;
  P->budget = c.budget_bytes ? c.budget_bytes : (free_b > margin ? free_b - margin : free_b / 2);
  P->chunk_bytes = c.staging_chunk_bytes ? ((c.staging_chunk_bytes + 4095) & ~size_t(4095)) : (size_t(64) << 20);
  const int nchunks = c.staging_chunks > 0 ? c.staging_chunks : 4;
  SAGE_CK(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
  SAGE_CK(cudaStreamCreateWithFlags(&P->alloc, cudaStreamNonBlocking));
  {
    cudaError_t he = cudaSuccess;
    P->ring_mem = static_cast<char*>(host_alloc_pinned(P->chunk_bytes * nchunks, &he));
    if (!P->ring_mem)
      return fail(SAGE_ERR_NOMEM, "pinned staging ring of %zu bytes: %s", P->chunk_bytes * nchunks,
                  cudaGetErrorString(he));
  }
  for (int i = 0; i < nchunks; ++i) {
    P->ring.push_back(P->ring_mem + static_cast<size_t>(i) * P->chunk_bytes);
    cudaEvent_t ev;
    SAGE_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SAGE_CK(cudaEventRecord(ev, P->side));
    P->ring_ev.push_back(ev);
  }
  int hw = static_cast<int>(std::thread::hardware_concurrency());
  int nthreads = c.producer_threads > 0 ? c.producer_threads : std::min(16, std::max(1, hw));
  P->workers.reset(new Workers(std::max(0, nthreads - 1)));
  sage_pool_s* raw = P.get();
  P->stager = std::thread([raw] { stager_loop(raw); });
  P->st.ctx_ms = ms_since(t0);
  *out = P.release();
  return SAGE_OK;
}

// sage_prepare on local data sources (imp == nullptr), or on read-only items
// mapped from the owning process (imp; see prepare_imported).  The descriptor
// has been checked.
static sage_status prepare_impl(sage_pool P, const sage_fn_desc* d, sage_fn* out,
                                std::unique_ptr<sage::ImportedData> imp) {
  *out = nullptr;
  sage_status st = SAGE_OK;
  auto t0 = Clock::now();
  SAGE_CK(cudaSetDevice(P->device));
  Entry* e = nullptr;
  {
    std::lock_guard<std::mutex> g(P->mu);
    P->st.prepares++;
    auto it = P->entries.find(d->fn_key);
    if (it != P->entries.end()) {
      // read-only sharing: take a reference, load nothing
      if (!same_shape(it->second, d))
        return fail(SAGE_ERR_INVALID, "key '%s' is resident with another shape", d->fn_key);
      it->second->refs++;
      P->st.hits++;
      imp.reset();  // this process already holds the key: the extra mapping goes back
      sage_fn f = new sage_fn_s{P, it->second, kFnMagic};
      P->handles.insert(f);
      *out = f;
      P->st.last_prepare_ms = ms_since(t0);
      return SAGE_OK;
    }
    e = new Entry();
    e->pool = P;
    e->key = d->fn_key;
    e->dtype = d->dtype;
    e->T = d->num_tables;
    e->dim = d->dim;
    e->n_dense = d->n_dense;
    e->rows.assign(d->rows, d->rows + d->num_tables);
    e->bot.assign(d->bot_dims, d->bot_dims + d->n_bot);
    e->top.assign(d->top_dims, d->top_dims + d->n_top);
    e->tables_bytes = d->tables.bytes;
    e->weights_bytes = d->weights.bytes;
    e->tdesc = d->tables;
    e->wdesc = d->weights;
    e->sig = shape_sig(d);
    e->imp = std::move(imp);
    if (!e->imp) {
      auto hc = P->hcache.find(e->key);
      if (hc != P->hcache.end() && hc->second.sig == e->sig) {
        // re-stage from the host image (stage 2 -> resident): no producer call
        e->owned = hc->second;
        P->hcache.erase(hc);
        e->tdesc.host_src = e->owned.tables;
        e->tdesc.fill = nullptr;
        e->wdesc.host_src = e->owned.weights;
        e->wdesc.fill = nullptr;
        P->st.host_cache_hits++;
      }
    }
    e->max_batch = d->max_batch > 0 ? d->max_batch : 4096;
    if (e->dtype == SAGE_F32) {
      // pre-split planes when every hidden layer runs on the tensor cores
      std::vector<std::pair<int, int>> dims;
      int prev = e->n_dense;
      for (int v : e->bot) dims.push_back({prev, v}), prev = v;
      prev = e->concat_dim();
      for (int v : e->top) dims.push_back({prev, v}), prev = v;
      bool all = dims.size() > 2;
      for (size_t l = 1; l + 1 < dims.size(); ++l)
        all = all && f32_on_tensor_cores(dims[l].second, dims[l].first, dims[l].first, dims[l].second) &&
              (e->concat_dim() % 4) == 0;
      e->presplit = all;
      if (all)
        for (size_t l = 1; l + 1 < dims.size(); ++l)
          e->wsplit_bytes += 2 * align256(static_cast<size_t>(dims[l].first) * dims[l].second * 4);
    }
    const int nslots = d->workspace_slots > 0 ? d->workspace_slots : 2;
    e->slots.resize(nslots);
    e->ws_bytes = static_cast<size_t>(nslots) * slot_bytes(e, e->max_batch);
    // an imported copy is the owner's memory: only this process's workspace counts here
    const size_t ro = e->imp ? 0 : align256(e->tables_bytes) + align256(e->weights_bytes);
    const size_t need = ro + e->ws_bytes + e->wsplit_bytes + 256;
    if (P->used + need > P->budget) {
      delete e;
      return fail(SAGE_ERR_NOMEM, "prepare of '%s' needs %zu bytes; %zu of %zu in use", d->fn_key, need, P->used,
                  P->budget);
    }
    P->used += need;
    e->reserved = need;
    e->refs = 1;
    e->t_prepare = t0;
    P->entries[e->key] = e;
    P->st.misses++;
  }
  auto setup_failed = [&](sage_status s2) {
    std::string msg = t_err;
    {
      std::lock_guard<std::mutex> g(e->smu);
      e->setup = 2;
      if (!e->queued) e->sstate = 2;
      e->scv.notify_all();
    }
    bool last = false;
    {
      std::lock_guard<std::mutex> g(P->mu);
      auto it = P->entries.find(e->key);
      if (it != P->entries.end() && it->second == e) P->entries.erase(it);
      last = --e->refs == 0;
    }
    if (last) destroy_entry(P, e);
    t_err = msg;
    return s2;
  };

  // read-only copy and the staging job (returns at once)
  cudaError_t ce = cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    e->ready = nullptr;
    return setup_failed(fail(SAGE_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(ce)));
  }
  if (e->imp) {
    e->d_tables = e->imp->tables;
    e->d_weights = e->imp->weights;
  } else {
    e->d_tables = static_cast<char*>(P->ro_alloc(e->tables_bytes, P->alloc));
    e->d_weights = static_cast<char*>(P->ro_alloc(e->weights_bytes, P->alloc));
  }
  if (!e->d_tables || !e->d_weights)
    return setup_failed(fail(SAGE_ERR_NOMEM, "device allocation of the read-only data of '%s' failed", d->fn_key));
  if (e->wsplit_bytes) {
    e->d_wsplit = static_cast<char*>(P->dev_alloc(e->wsplit_bytes, P->alloc));
    if (!e->d_wsplit) return setup_failed(fail(SAGE_ERR_NOMEM, "split-weight allocation failed"));
  }
  {
    // layer pointers inside the weights item (and the split planes of the hidden layers)
    size_t o = 0, ow = 0;
    int prev = e->n_dense;
    std::vector<std::pair<int, int>> L;
    for (int v : e->bot) {
      L.push_back({prev, v});
      prev = v;
    }
    prev = e->concat_dim();
    for (int v : e->top) {
      L.push_back({prev, v});
      prev = v;
    }
    for (size_t l = 0; l < L.size(); ++l) {
      const auto& p = L[l];
      o = align256(o);
      const void* W = e->d_weights + o;
      o += static_cast<size_t>(p.first) * p.second * e->elem();
      o = align256(o);
      const float* b = reinterpret_cast<const float*>(e->d_weights + o);
      o += static_cast<size_t>(p.second) * 4;
      e->layers.push_back({p.first, p.second, W, b});
      if (e->presplit && l >= 1 && l + 1 < L.size()) {
        const size_t pb = align256(static_cast<size_t>(p.first) * p.second * 4);
        e->wplanes.push_back({reinterpret_cast<const float*>(e->d_wsplit + ow),
                              reinterpret_cast<const float*>(e->d_wsplit + ow + pb)});
        ow += 2 * pb;
      } else {
        e->wplanes.push_back({nullptr, nullptr});
      }
    }
  }
  // the staging copies (side stream) may target the slab only once it exists
  ce = cudaStreamSynchronize(P->alloc);
  if (ce != cudaSuccess) return setup_failed(fail(SAGE_ERR_CUDA, "allocation: %s", cudaGetErrorString(ce)));
  {
    int64_t o = 0;
    for (int t = 0; t < e->T; ++t) {
      e->table_off[t] = o;
      o += e->rows[t] * e->dim * static_cast<int64_t>(e->elem());
    }
  }
  {
    std::lock_guard<std::mutex> g(e->smu);
    e->queued = true;  // the read-only items exist from here on
    e->scv.notify_all();
  }
  if (e->imp) {
    // the owner stages; this process only waits for its word, then opens the gate
    e->imp_waiter = std::thread([P, e] {
      cudaSetDevice(P->device);
      const bool ok = e->imp->wait_ready();
      finish_staging(P, e, ok, 0.0);
    });
  } else {
    {
      std::lock_guard<std::mutex> g(P->qmu);
      P->queue.push_back(e);
    }
    P->qcv.notify_one();
  }
  if (P->serial_setup) {
    std::unique_lock<std::mutex> l(e->smu);
    e->scv.wait(l, [&] { return e->sstate != 0; });
    l.unlock();
    cudaEventSynchronize(e->ready);
  }

  // meanwhile on this thread: kernels (module load) and workspace
  auto tm = Clock::now();
  load_kernels_once();
  const double module_ms = ms_since(tm);
  auto tw = Clock::now();
  e->d_err = static_cast<int*>(P->dev_alloc(256, P->alloc));
  if (!e->d_err) return setup_failed(fail(SAGE_ERR_NOMEM, "error word allocation failed"));
  ce = cudaMemsetAsync(e->d_err, 0, 256, P->alloc);
  if (ce != cudaSuccess) return setup_failed(fail(SAGE_ERR_CUDA, "memset: %s", cudaGetErrorString(ce)));
  for (auto& s : e->slots) {
    st = build_slot(e, s, e->max_batch, P->alloc);
    if (st != SAGE_OK) return setup_failed(st);
    ce = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s.branch, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s.h2d, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s.capture, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&s.copied, cudaEventDisableTiming);
    if (ce != cudaSuccess) return setup_failed(fail(SAGE_ERR_CUDA, "event: %s", cudaGetErrorString(ce)));
  }
  // allocations on the side stream must precede any use on other streams
  ce = cudaStreamSynchronize(P->alloc);
  if (ce != cudaSuccess) return setup_failed(fail(SAGE_ERR_CUDA, "setup sync: %s", cudaGetErrorString(ce)));
  const double ws_ms = ms_since(tw);
  {
    std::lock_guard<std::mutex> g(e->smu);
    e->setup = 1;
    e->scv.notify_all();
  }
  sage_fn f = new sage_fn_s{P, e, kFnMagic};
  {
    std::lock_guard<std::mutex> g(P->mu);
    P->handles.insert(f);
    P->st.last_module_ms = module_ms;
    P->st.last_workspace_ms = ws_ms;
    P->st.last_prepare_ms = ms_since(t0);
  }
  *out = f;
  return SAGE_OK;
}

sage_status sage_prepare(sage_pool P, const sage_fn_desc* d, sage_fn* out) {
  if (!P || !out) return fail(SAGE_ERR_INVALID, "null pool or out");
  *out = nullptr;
  sage_status st = check_desc(d);
  if (st != SAGE_OK) return st;
  return prepare_impl(P, d, out, nullptr);
}

sage_status sage_fn_data(sage_fn f, const void** tables, const void** weights) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  if (tables) *tables = f->e->d_tables;
  if (weights) *weights = f->e->d_weights;
  return SAGE_OK;
}

sage_status sage_fn_query(sage_fn f) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  Entry* e = f->e;
  std::unique_lock<std::mutex> l(e->smu);
  if (e->sstate == 2) return fail(SAGE_ERR_STAGING, "staging of '%s' failed", e->key.c_str());
  if (e->setup == 2) return fail(SAGE_ERR_CUDA, "setup of '%s' failed", e->key.c_str());
  if (e->sstate == 0 || e->setup == 0) return SAGE_PENDING;
  cudaEvent_t ev = e->ready;
  l.unlock();
  cudaError_t q = cudaEventQuery(ev);
  if (q == cudaSuccess) return SAGE_OK;
  if (q == cudaErrorNotReady) {
    cudaGetLastError();
    return SAGE_PENDING;
  }
  return fail(SAGE_ERR_CUDA, "cudaEventQuery: %s", cudaGetErrorString(q));
}

sage_status sage_wait(sage_fn f, int64_t timeout_us) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  auto t0 = Clock::now();
  for (;;) {
    sage_status st = sage_fn_query(f);
    if (st != SAGE_PENDING) return st;
    if (timeout_us >= 0 &&
        std::chrono::duration<double, std::micro>(Clock::now() - t0).count() > static_cast<double>(timeout_us))
      return fail(SAGE_ERR_TIMEOUT, "staging of '%s' not finished within %lld us", f->e->key.c_str(),
                  static_cast<long long>(timeout_us));
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

sage_status sage_invoke_batch(sage_fn f, const sage_invocation* invs, int n, void* stream) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  if (n < 0 || (n > 0 && !invs)) return fail(SAGE_ERR_INVALID, "bad invocation list");
  Entry* e = f->e;
  sage_status st = wait_ready_enqueued(e);
  if (st != SAGE_OK) return st;
  SAGE_CK(cudaSetDevice(e->pool->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<InvTable> tab(new InvTable());
  int i = 0;
  while (i < n) {
    tab->n = 0;
    int64_t M = 0;
    while (i < n && tab->n < kMaxInv) {
      const sage_invocation& v = invs[i];
      if (v.batch < 0) return fail(SAGE_ERR_INVALID, "invocation %d: negative batch", i);
      if (v.batch > 0 && (!v.dense || !v.indices || !v.offsets || !v.out))
        return fail(SAGE_ERR_INVALID, "invocation %d: null buffer", i);
      if (M + v.batch > (int64_t(1) << 30)) return fail(SAGE_ERR_INVALID, "batch too large (over 2^30 rows)");
      if (v.batch > 0) {
        InvDesc& dd = tab->d[tab->n++];
        dd.dense = v.dense;
        dd.indices = v.indices;
        dd.offsets = v.offsets;
        dd.out = v.out;
        dd.batch = v.batch;
        dd.row_base = static_cast<int>(M);
        dd.nidx = v.num_indices;
        M += v.batch;
      }
      ++i;
    }
    tab->M = static_cast<int>(M);
    if (tab->n == 0) continue;
    index_invocations(*tab);
    st = run_batch(e, *tab, s);
    if (st != SAGE_OK) return st;
    e->pool->invocations += tab->n;
  }
  return SAGE_OK;
}

sage_status sage_invoke(sage_fn f, const sage_invocation* inv, void* stream) {
  if (!inv) return fail(SAGE_ERR_INVALID, "null invocation");
  return sage_invoke_batch(f, inv, 1, stream);
}

}  // extern "C"

namespace sage {

sage_status check_shape(const sage_fn_desc* d) { return check_shape_impl(d); }

int pool_device(sage_pool P) { return P ? P->device : 0; }

bool pool_exportable(sage_pool P) { return P && P->exportable; }

std::string shape_signature(const sage_fn_desc* d) { return shape_sig(d); }

sage_status prepare_imported(sage_pool P, const sage_fn_desc* d, ImportedData* imp, sage_fn* out) {
  std::unique_ptr<ImportedData> own(imp);
  if (!P || !out || !imp) return fail(SAGE_ERR_INVALID, "null pool, out or import");
  *out = nullptr;
  sage_status st = check_shape_impl(d);
  if (st != SAGE_OK) return st;
  return prepare_impl(P, d, out, std::move(own));
}

sage_status fn_export(sage_fn f, VmmBlock* tables, VmmBlock* weights) {
  if (!valid_fn(f) || !tables || !weights) return fail(SAGE_ERR_INVALID, "invalid function handle");
  sage_pool_s* P = f->pool;
  if (!P->exportable) return fail(SAGE_ERR_INVALID, "the pool was not created exportable");
  Entry* e = f->e;
  {
    // a handle shared from a concurrent first prepare may precede the allocation
    std::unique_lock<std::mutex> l(e->smu);
    e->scv.wait(l, [&] { return e->queued || e->sstate == 2 || e->setup == 2; });
    if (!e->queued) return fail(SAGE_ERR_STAGING, "setup of '%s' failed", e->key.c_str());
  }
  std::lock_guard<std::mutex> g(P->mu);
  auto t = P->vmm.find(f->e->d_tables);
  auto w = P->vmm.find(f->e->d_weights);
  if (t == P->vmm.end() || w == P->vmm.end()) return fail(SAGE_ERR_INVALID, "read-only data is not exportable");
  *tables = t->second;
  *weights = w->second;
  return SAGE_OK;
}

bool host_csr_valid(const sage_host_invocation& v, int T) {
  if (v.batch <= 0) return true;
  if (!v.offsets || T < 1) return false;
  const size_t nb = static_cast<size_t>(T) * v.batch;
  const int64_t* o = v.offsets;
  if (o[0] != 0 || o[nb] != v.num_indices) return false;
  bool bad = false;  // one pass without early exit: the compiler vectorises it
  for (size_t j = 0; j < nb; ++j) bad |= o[j + 1] < o[j];
  return !bad;
}

}  // namespace sage


// Fused batch from host buffers, asynchronous on `stream`: merged H2D copies of
// the inputs into the slot's I/O arena, the launch chain, merged D2H copies of the
// outputs.  slot >= 0 pins the workspace slot (the serving loop gives each of its
// lanes its own slot); -1 takes the next slot in turn.
sage_status sage::host_batch_async(sage_fn f, const sage_host_invocation* invs, int n, cudaStream_t s, int slot) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  if (n < 0 || (n > 0 && !invs)) return fail(SAGE_ERR_INVALID, "bad invocation list");
  if (n > kMaxInv) return fail(SAGE_ERR_INVALID, "more than %d invocations in one host batch", kMaxInv);
  Entry* e = f->e;
  sage_status st = wait_ready_enqueued(e);
  if (st != SAGE_OK) return st;
  SAGE_CK(cudaSetDevice(e->pool->device));
  // arena regions: dense | indices | offsets | out, each invocation's part 256-aligned
  size_t nd = 0, ni = 0, no = 0, nu = 0;
  int64_t M = 0;
  for (int i = 0; i < n; ++i) {
    const sage_host_invocation& v = invs[i];
    if (v.batch < 0 || v.num_indices < 0) return fail(SAGE_ERR_INVALID, "invocation %d: bad sizes", i);
    if (v.batch == 0) continue;
    if (!v.dense || !v.offsets || !v.out || (v.num_indices > 0 && !v.indices))
      return fail(SAGE_ERR_INVALID, "invocation %d: null buffer", i);
    if (!host_csr_valid(v, e->T))
      return fail(SAGE_ERR_INVALID, "invocation %d: offsets must start at 0, never decrease and end at num_indices",
                  i);
    nd +=static_cast<size_t>(v.batch) * e->n_dense * 4;
    ni += static_cast<size_t>(v.num_indices) * 4;
    no += (static_cast<size_t>(e->T) * v.batch + 1) * 8;
    nu += static_cast<size_t>(v.batch) * 4;
    M += v.batch;
  }
  if (M == 0) return SAGE_OK;
  const size_t need = align256(nd) + align256(ni) + align256(no) + align256(nu);
  std::unique_ptr<InvTable> tab(new InvTable());
  {
    std::lock_guard<std::mutex> g(e->imu);
    Slot* sl = nullptr;
    st = acquire_slot(e, static_cast<int>(M), s, &sl, slot);
    if (st != SAGE_OK) return st;
    if (sl->io_bytes < need) {
      if (sl->used) SAGE_CK(cudaEventSynchronize(sl->done));
      e->pool->dev_free(sl->io, sl->io_bytes, s);
      const size_t nb = need + need / 4;
      sl->io = static_cast<char*>(e->pool->dev_alloc(nb, s));
      sl->io_bytes = sl->io ? nb : 0;
      if (!sl->io) return fail(SAGE_ERR_NOMEM, "host-invocation arena of %zu bytes", nb);
      // the copy stream may use the new arena only after its allocation on `s`
      SAGE_CK(cudaEventRecord(sl->copied, s));
      SAGE_CK(cudaStreamWaitEvent(sl->h2d, sl->copied, 0));
    }
    char* pd = sl->io;
    char* pi = pd + align256(nd);
    char* po = pi + align256(ni);
    char* pu = po + align256(no);
    // H2D copies; adjacent host ranges are merged into one copy
    struct Run {
      char* dst;
      const char* src;
      size_t n;
    };
    std::vector<Run> runs;
    auto add = [&](char* dst, const void* src, size_t nbytes) {
      if (nbytes == 0) return;
      if (!runs.empty() && runs.back().dst + runs.back().n == dst &&
          runs.back().src + runs.back().n == static_cast<const char*>(src)) {
        runs.back().n += nbytes;
      } else {
        runs.push_back({dst, static_cast<const char*>(src), nbytes});
      }
    };
    tab->n = 0;
    int64_t row = 0;
    std::vector<Run> dense_r, idx_r, off_r;
    size_t od = 0, oi = 0, oo = 0, ou = 0;
    for (int i = 0; i < n; ++i) {
      const sage_host_invocation& v = invs[i];
      if (v.batch == 0) continue;
      const size_t bd = static_cast<size_t>(v.batch) * e->n_dense * 4;
      const size_t bi = static_cast<size_t>(v.num_indices) * 4;
      const size_t bo = (static_cast<size_t>(e->T) * v.batch + 1) * 8;
      InvDesc& dd = tab->d[tab->n++];
      dd.dense = reinterpret_cast<const float*>(pd + od);
      dd.indices = reinterpret_cast<const int32_t*>(pi + oi);
      dd.offsets = reinterpret_cast<const int64_t*>(po + oo);
      dd.out = reinterpret_cast<float*>(pu + ou);
      dd.batch = v.batch;
      dd.row_base = static_cast<int>(row);
      dd.nidx = v.num_indices;
      dense_r.push_back({pd + od, reinterpret_cast<const char*>(v.dense), bd});
      idx_r.push_back({pi + oi, reinterpret_cast<const char*>(v.indices), bi});
      off_r.push_back({po + oo, reinterpret_cast<const char*>(v.offsets), bo});
      od += bd;
      oi += bi;
      oo += bo;
      ou += static_cast<size_t>(v.batch) * 4;
      row += v.batch;
    }
    tab->M = static_cast<int>(row);
    index_invocations(*tab);
    for (auto& r : dense_r) add(r.dst, r.src, r.n);
    for (auto& r : idx_r) add(r.dst, r.src, r.n);
    for (auto& r : off_r) add(r.dst, r.src, r.n);
    if (sl->used) SAGE_CK(cudaStreamWaitEvent(sl->h2d, sl->done, 0));
    for (auto& r : runs) SAGE_CK(cudaMemcpyAsync(r.dst, r.src, r.n, cudaMemcpyHostToDevice, sl->h2d));
    SAGE_CK(cudaEventRecord(sl->copied, sl->h2d));
    SAGE_CK(cudaStreamWaitEvent(s, sl->copied, 0));
    SAGE_CK(cudaStreamWaitEvent(s, e->ready, 0));
    // direct launches: replaying the chain as a CUDA graph (capture + update per batch)
    // measured slower here, where the host's time per batch is on the critical path
    st = launch_chain(e, *sl, *tab, s, sage::stream_is_confined(s));
    if (st != SAGE_OK) return st;
    // D2H of the outputs, merged where the host outputs are adjacent
    runs.clear();
    size_t ou2 = 0;
    for (int i = 0; i < n; ++i) {
      const sage_host_invocation& v = invs[i];
      if (v.batch == 0) continue;
      const size_t bu = static_cast<size_t>(v.batch) * 4;
      char* hdst = reinterpret_cast<char*>(v.out);
      if (!runs.empty() && const_cast<char*>(runs.back().src) + runs.back().n == pu + ou2 &&
          runs.back().dst + runs.back().n == hdst) {
        runs.back().n += bu;
      } else {
        runs.push_back({hdst, pu + ou2, bu});
      }
      ou2 += bu;
    }
    for (auto& r : runs) SAGE_CK(cudaMemcpyAsync(r.dst, r.src, r.n, cudaMemcpyDeviceToHost, s));
    SAGE_CK(cudaEventRecord(sl->done, s));
    sl->used = true;
  }
  e->pool->invocations += n;
  return SAGE_OK;
}

extern "C" {

sage_status sage_invoke_batch_host_async(sage_fn f, const sage_host_invocation* invs, int n, void* stream) {
  if (n < 0 || (n > 0 && !invs)) return fail(SAGE_ERR_INVALID, "bad invocation list");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; i += kMaxInv) {
    sage_status st = sage::host_batch_async(f, invs + i, std::min(kMaxInv, n - i), s, -1);
    if (st != SAGE_OK) return st;
  }
  return SAGE_OK;
}

sage_status sage_invoke_batch_host(sage_fn f, const sage_host_invocation* invs, int n, void* stream) {
  if (n < 0 || (n > 0 && !invs)) return fail(SAGE_ERR_INVALID, "bad invocation list");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; i += kMaxInv) {
    sage_status st = sage::host_batch_async(f, invs + i, std::min(kMaxInv, n - i), s, -1);
    if (st != SAGE_OK) return st;
  }
  SAGE_CK(cudaStreamSynchronize(s));
  return SAGE_OK;
}


sage_status sage_autotune(sage_fn f, int rows, void* stream) {
  if (!valid_fn(f) || rows < 1) return fail(SAGE_ERR_INVALID, "bad autotune arguments");
  Entry* e = f->e;
  SAGE_CK(cudaSetDevice(e->pool->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = static_cast<int>(e->bot.size()), nl = static_cast<int>(e->layers.size());
  for (int l = 1; l + 1 < nl; ++l) {
    const Layer& L = e->layers[l];
    int kind = 0;
    if (e->dtype == SAGE_BF16) {
      kind = kGemmBf16;
    } else {
      const int ldx = l < nb ? L.in : (l == nb ? e->concat_dim() : L.in);
      const int ldy = l == nb - 1 ? e->concat_dim() : L.out;
      if (e->presplit) kind = kGemmTf32Pre;
      else if (f32_on_tensor_cores(L.out, L.in, ldx, ldy)) kind = kGemmTf32x3;
    }
    if (!kind) continue;
    sage_status st = autotune_gemm(kind, rows, L.out, L.in, s, nullptr, nullptr);
    if (st != SAGE_OK) return st;
  }
  if (e->presplit && nb >= 2 && bottom01_fusable(e->layers[0].in, e->layers[0].out, e->layers[1].out))
    return autotune_bottom01(rows, e->layers[0].in, e->layers[0].out, e->layers[1].out,
                             nb >= 3 ? e->layers[2].out : 0, s, nullptr);
  return SAGE_OK;
}

sage_status sage_fn_check(sage_fn f) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  Entry* e = f->e;
  sage_status st = wait_ready_enqueued(e);
  if (st != SAGE_OK) return st;
  SAGE_CK(cudaSetDevice(e->pool->device));
  {
    std::lock_guard<std::mutex> g(e->imu);
    for (auto& s : e->slots)
      if (s.used) SAGE_CK(cudaEventSynchronize(s.done));
  }
  int w = 0;
  SAGE_CK(cudaMemcpy(&w, e->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  SAGE_CK(cudaMemset(e->d_err, 0, sizeof(int)));
  if (w & kErrTimeout) {
    // a kernel that gave up may have left fused-head arrival counters short
    std::lock_guard<std::mutex> g(e->imu);
    for (auto& s : e->slots) {
      if (s.hcnt) SAGE_CK(cudaMemset(s.hcnt, 0, static_cast<size_t>(s.cap) * 4));
      if (s.gwork) SAGE_CK(cudaMemset(s.gwork, 0, 2 * sizeof(unsigned)));
    }
  }
  if (w & kErrTimeout) return fail(SAGE_ERR_DEVICE, "a kernel's bounded wait ran out");
  if (w & kErrBounds) return fail(SAGE_ERR_BOUNDS, "a bag row index was outside its table");
  return SAGE_OK;
}

sage_status sage_fn_debug_copy(sage_fn f, int which, int plane, void* dst, size_t bytes, int* rows_out) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  Entry* e = f->e;
  std::lock_guard<std::mutex> g(e->imu);
  if (e->last_slot < 0) return fail(SAGE_ERR_INVALID, "no batch has run on this function");
  const int M = e->last_M;
  if (rows_out) *rows_out = M;
  if (!dst) return SAGE_OK;
  Slot& s = e->slots[e->last_slot];
  const int nt = static_cast<int>(e->top.size());
  const char* buf = nullptr;
  int width = 0;
  if (which == 0) {
    if (!s.pooled_written)
      return fail(SAGE_ERR_INVALID, "the pooled columns are not written (the gather ran fused with the first top "
                                    "layer; tuning kind 5 set to (1, 1) keeps them)");
    buf = s.concat;
    width = e->concat_dim();
  } else if (which >= 1 && which < nt) {
    if (which > s.top_written)
      return fail(SAGE_ERR_INVALID, "top hidden layer %d is not written (the head runs in its epilogue)", which - 1);
    buf = s.top[which - 1];
    width = e->top[which - 1];
  } else {
    return fail(SAGE_ERR_INVALID, "buffer %d does not exist", which);
  }
  if (plane < 0 || plane >= static_cast<int>(planes(e))) return fail(SAGE_ERR_INVALID, "plane %d does not exist", plane);
  const size_t need = static_cast<size_t>(M) * width * e->elem();
  if (bytes != need) return fail(SAGE_ERR_INVALID, "bytes %zu != %zu", bytes, need);
  if (plane == 1) buf += static_cast<size_t>(s.cap) * width * e->elem();
  SAGE_CK(cudaSetDevice(e->pool->device));
  if (s.used) SAGE_CK(cudaEventSynchronize(s.done));
  SAGE_CK(cudaMemcpy(dst, buf, need, cudaMemcpyDeviceToHost));
  return SAGE_OK;
}

sage_status sage_release(sage_fn f) {
  if (!valid_fn(f)) return fail(SAGE_ERR_INVALID, "invalid function handle");
  sage_pool_s* P = f->pool;
  Entry* e = nullptr;
  {
    std::lock_guard<std::mutex> g(P->mu);
    auto it = P->handles.find(f);
    if (it == P->handles.end()) return fail(SAGE_ERR_INVALID, "handle already released");
    P->handles.erase(it);
    f->magic = 0;
    if (--f->e->refs == 0) {
      e = f->e;
      auto ie = P->entries.find(e->key);
      if (ie != P->entries.end() && ie->second == e) P->entries.erase(ie);
    }
  }
  delete f;
  if (e) {
    SAGE_CK(cudaSetDevice(P->device));
    const cudaError_t ce = destroy_entry(P, e);
    if (ce != cudaSuccess)
      return fail(SAGE_ERR_CUDA, "released, but work of the function had failed on the device: %s",
                  cudaGetErrorString(ce));
  }
  return SAGE_OK;
}

sage_status sage_pool_destroy(sage_pool P) {
  if (!P) return fail(SAGE_ERR_INVALID, "null pool");
  {
    std::lock_guard<std::mutex> g(P->mu);
    if (!P->handles.empty()) return fail(SAGE_ERR_BUSY, "%zu function handles are live", P->handles.size());
  }
  {
    std::lock_guard<std::mutex> g(P->qmu);
    P->stop = true;
  }
  P->qcv.notify_all();
  if (P->stager.joinable()) P->stager.join();
  cudaSetDevice(P->device);
  cudaError_t ce = cudaStreamSynchronize(P->side);
  const cudaError_t ce2 = cudaStreamSynchronize(P->alloc);
  if (ce == cudaSuccess) ce = ce2;
  for (auto& kv : P->hcache) free_image(P, kv.second);
  P->hcache.clear();
  for (size_t i = 0; i < P->ring.size(); ++i) {
    cudaEventDestroy(P->ring_ev[i]);
  }
  host_free_pinned(P->ring_mem);
  cudaStreamDestroy(P->side);
  cudaStreamDestroy(P->alloc);
  P->workers.reset();
  delete P;
  if (ce != cudaSuccess)
    return fail(SAGE_ERR_CUDA, "pool destroyed, but its staging work had failed on the device: %s",
                cudaGetErrorString(ce));
  return SAGE_OK;
}

sage_status sage_pool_stats(sage_pool P, sage_pool_stats_t* out) {
  if (!P || !out) return fail(SAGE_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> g(P->mu);
  sage_pool_stats_t s = P->st;
  s.budget_bytes = P->budget;
  s.resident_bytes = P->used;
  s.readonly_bytes = 0;
  s.functions = static_cast<int64_t>(P->entries.size());
  s.refs = static_cast<int64_t>(P->handles.size());
  for (auto& kv : P->entries) s.readonly_bytes += kv.second->tables_bytes + kv.second->weights_bytes;
  s.host_cache_bytes = 0;
  for (auto& kv : P->hcache) s.host_cache_bytes += kv.second.bytes();
  s.host_cache_entries = static_cast<int64_t>(P->hcache.size());
  s.h2d_bytes = P->h2d.load();
  s.invocations = P->invocations.load();
  s.launches = sage::launches();
  *out = s;
  return SAGE_OK;
}

// ---------------------------------------------------------------- building blocks

sage_status sage_embedding_bag_sum(sage_dtype dtype, const void* tables, const int64_t* table_rows, int num_tables,
                                   int dim, int batch, const int32_t* indices, const int64_t* offsets, void* out,
                                   int ldo, int* err_word, void* stream) {
  if (num_tables < 1 || num_tables > kMaxTables || !tables || !table_rows || batch < 0 || !out)
    return fail(SAGE_ERR_INVALID, "bad embedding-bag arguments");
  if (batch == 0) return SAGE_OK;
  const int es = dtype == SAGE_BF16 ? 2 : 4;
  if (ldo < num_tables * dim || ((static_cast<size_t>(ldo) * es) & 15) || (reinterpret_cast<uintptr_t>(out) & 15) ||
      (reinterpret_cast<uintptr_t>(tables) & 15))
    return fail(SAGE_ERR_INVALID, "ldo / alignment");
  std::unique_ptr<InvTable> tab(new InvTable());
  tab->n = 1;
  tab->M = batch;
  tab->d[0] = InvDesc{nullptr, indices, offsets, nullptr, batch, 0, 0};
  GatherArgs a;
  a.dtype = dtype;
  a.tables = static_cast<const char*>(tables);
  int64_t o = 0;
  for (int t = 0; t < num_tables; ++t) {
    if (table_rows[t] < 1 || table_rows[t] >= (int64_t(1) << 31)) return fail(SAGE_ERR_INVALID, "bad table_rows");
    a.table_off[t] = o;
    a.table_rows[t] = static_cast<int32_t>(table_rows[t]);
    o += table_rows[t] * dim * es;
  }
  a.T = num_tables;
  a.dim = dim;
  a.out = out;
  a.ldo = ldo;
  a.err = err_word;
  cudaError_t e = launch_gather(a, *tab, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(SAGE_ERR_INVALID, "unsupported dim");
  SAGE_CK(e);
  return SAGE_OK;
}

sage_status sage_linear(sage_dtype dtype, int M, int N, int K, const void* x, int ldx, const void* W,
                        const float* bias, int act, void* y, int ldy, int* err_word, void* stream) {
  if (M < 0 || N < 1 || K < 1 || !x || !W || !bias || !y) return fail(SAGE_ERR_INVALID, "bad linear arguments");
  cudaError_t e;
  if (dtype == SAGE_BF16)
    e = launch_linear_bf16_tc(M, N, K, x, ldx, W, bias, act, y, ldy, err_word, static_cast<cudaStream_t>(stream),
                              tuned_gemm(kGemmBf16, M, N, K));
  else
    e = launch_f32_layer(M, N, K, static_cast<const float*>(x), ldx, static_cast<const float*>(W), bias, act,
                         static_cast<float*>(y), ldy, err_word, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return fail(SAGE_ERR_INVALID, "unsupported shape or alignment");
  SAGE_CK(e);
  return SAGE_OK;
}

sage_status sage_linear_tiled(sage_dtype dtype, int M, int N, int K, const void* x, int ldx, const void* W,
                              const float* bias, int act, void* y, int ldy, int bn, int stages, int* err_word,
                              void* stream) {
  if (bn == 0 && stages == 0) return sage_linear(dtype, M, N, K, x, ldx, W, bias, act, y, ldy, err_word, stream);
  if (M < 0 || N < 1 || K < 1 || !x || !W || !bias || !y) return fail(SAGE_ERR_INVALID, "bad linear arguments");
  GemmCfg cands[16];
  const int nc = gemm_candidates(dtype == SAGE_BF16 ? kGemmBf16 : kGemmTf32x3, cands, 16);
  bool known = false;
  for (int c = 0; c < nc; ++c) known |= cands[c].bn == bn && cands[c].stages == stages;
  if (!known) return fail(SAGE_ERR_INVALID, "unknown tile configuration (%d, %d)", bn, stages);
  cudaError_t e;
  if (dtype == SAGE_BF16)
    e = launch_linear_bf16_tc(M, N, K, x, ldx, W, bias, act, y, ldy, err_word, static_cast<cudaStream_t>(stream),
                              GemmCfg{bn, stages});
  else if (f32_on_tensor_cores(N, K, ldx, ldy))
    e = launch_linear_f32_tc(M, N, K, static_cast<const float*>(x), ldx, static_cast<const float*>(W), bias, act,
                             static_cast<float*>(y), ldy, err_word, static_cast<cudaStream_t>(stream),
                             GemmCfg{bn, stages});
  else
    return fail(SAGE_ERR_INVALID, "shape does not tile on the tensor cores");
  if (e == cudaErrorInvalidValue) return fail(SAGE_ERR_INVALID, "unsupported shape or alignment");
  SAGE_CK(e);
  return SAGE_OK;
}

}  // extern "C"
