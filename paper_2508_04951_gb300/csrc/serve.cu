// Serving loop with continuous batching (host C++; declared in include/dc.h).
//
// Requests (host pulses with their own fs, fc, v_r and TEC) are queued by
// dc_serve_submit.  One scheduler thread owns `slots` batch slots, each with
// its own stream, context and pinned staging.  The device memory of every
// batch in flight -- its input, its output and correct_batch's scratch --
// comes from one pool carved from the HBM budget at start (first fit, freed
// when the batch completes).  Whenever a slot is free and requests wait, the
// scheduler admits queued requests into it in arrival order while they fit
// the slot's staging and the pool can hold the batch; a request that the
// pool cannot hold yet waits for in-flight batches to finish (admission by
// HBM budget), one that finds every slot busy waits for a slot.  A launched
// batch runs H2D -> correct_batch -> D2H -> event on the slot's stream; the
// scheduler does not wait for the GPU, so the next slot fills with requests
// that arrive meanwhile and batches overlap on the device.  Completed slots
// (event query) hand results back to the callers' buffers, return their pool
// block and record the latency from submission to completion.  Where the
// device reads and writes pageable host memory through the host's page tables
// (GB300 with its Grace host), the batch's inputs and outputs move between
// the callers' buffers and the pool by copy kernels on the slot's stream
// (gather before correct_batch, scatter after it): no host copies, no
// staging, nothing on the scheduler thread; elsewhere (or with
// DC_SERVE_STAGED=1) host threads copy through pinned staging.  Each
// request's result does not depend on which batch it rode in (correct_batch's
// per-item independence).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dc.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id;
  const dc_c64* x;
  dc_c64* y;
  long long n;
  double fs, fc, v_r, tec;
  Clock::time_point t_submit, t_done;
  int state = 0;          // 0 queued, 1 in flight, 2 done, 3 failed, 4 cancelled
  dc_status status = DC_OK;
  bool waited_memory = false, waited_slot = false;
};

struct Slot {
  dc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  dc_c64* in_host = nullptr;    // pinned
  dc_c64* out_host = nullptr;   // pinned
  struct CopyChunk* chunks = nullptr;   // pinned: the gather / scatter lists (direct mode)
  long long cap = 0;            // samples of staging
  size_t block = 0, block_bytes = 0;   // this batch's pool block (offset, bytes)
  std::vector<Request*> reqs;
  std::vector<long long> offs;
  bool busy = false;
  bool direct_batch = false;    // this batch moves its data by copy kernels
};

// First-fit allocator over the device pool (offsets; 256-byte granules).
class PoolAlloc {
 public:
  void reset(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
    total_ = bytes;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
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
  size_t total() const { return total_; }
  size_t largest() const {
    size_t m = 0;
    for (const auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
  size_t peak() const { return peak_; }
  static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0, used_ = 0, peak_ = 0;
};

// Fixed pool of copy threads: parallel memcpy of request samples between
// callers' buffers and pinned staging (one thread moves ~10-15 GB/s; a
// request stream at 20 k pulses/s needs ~27 GB/s each way).
class CopyPool {
 public:
  explicit CopyPool(int n) {
    for (int i = 0; i < n; ++i) th_.emplace_back([this] { loop(); });
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  struct Job { void* dst; const void* src; size_t bytes; };
  // Copy all jobs, split into pieces of at most `piece` bytes; returns when done.
  void run(const std::vector<Job>& jobs, size_t piece = 1 << 20) {
    std::vector<Job> parts;
    for (const Job& j : jobs)
      for (size_t o = 0; o < j.bytes; o += piece)
        parts.push_back({(char*)j.dst + o, (const char*)j.src + o, std::min(piece, j.bytes - o)});
    {
      std::lock_guard<std::mutex> g(mu_);
      work_ = &parts;
      next_ = 0;
      left_ = parts.size();
    }
    cv_.notify_all();
    take_and_copy();                                   // the caller helps
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [this] { return left_ == 0; });
    work_ = nullptr;
  }

 private:
  bool take_and_copy() {
    bool any = false;
    while (true) {
      Job j;
      {
        std::lock_guard<std::mutex> g(mu_);
        if (!work_ || next_ >= work_->size()) break;
        j = (*work_)[next_++];
      }
      memcpy(j.dst, j.src, j.bytes);
      any = true;
      std::lock_guard<std::mutex> g(mu_);
      if (--left_ == 0) done_cv_.notify_all();
    }
    return any;
  }
  void loop() {
    std::unique_lock<std::mutex> lk(mu_);
    while (!stop_) {
      cv_.wait(lk, [this] { return stop_ || (work_ && next_ < work_->size()); });
      if (stop_) break;
      lk.unlock();
      take_and_copy();
      lk.lock();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<Job>* work_ = nullptr;
  size_t next_ = 0, left_ = 0;
  bool stop_ = false;
};

}  // namespace

struct dc_server {
  int device = 0;
  bool direct = false;          // gather / scatter kernels on the callers' buffers
  dc_opts opts{};
  std::vector<Slot> slots;
  long long cap = 0;            // samples per batch (staging)
  char* pool = nullptr;         // device pool: inputs, outputs, scratch of batches in flight
  PoolAlloc alloc;
  long long waited_memory = 0, waited_slot = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<long long, Request*> reqs;
  long long next_id = 1;
  bool stop = false;
  std::thread th;
  CopyPool* copies = nullptr;
  // statistics
  std::vector<double> latencies;
  long long done_samples = 0, completed = 0, batches = 0;
  Clock::time_point t_first{}, t_last{};
  bool have_first = false;
};

namespace {

// One chunk of a gather or scatter: n samples from src to dst (one side a
// caller's host buffer, read or written by the device through the host's page
// tables; the other the batch's block of the device pool).
struct CopyChunk {
  const dc_c64* src;
  dc_c64* dst;
  long long n;
};
constexpr int kCopyChunk = 16384;              // samples per chunk (one CTA)
constexpr int kMaxChunks = 65536;              // per slot and list (gather, scatter)

__global__ void __launch_bounds__(256) copy_chunks_kernel(const CopyChunk* __restrict__ list) {
  const CopyChunk c = list[blockIdx.x];
  const bool v4 = ((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst)) & 15) == 0;
  if (v4) {
    const float4* s4 = reinterpret_cast<const float4*>(c.src);
    float4* d4 = reinterpret_cast<float4*>(c.dst);
    for (long long i = threadIdx.x; i < c.n / 2; i += blockDim.x) d4[i] = s4[i];
    if ((c.n & 1) && threadIdx.x == 0) c.dst[c.n - 1] = c.src[c.n - 1];
  } else {
    for (long long i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.src[i];
  }
}

// The chunk list of a batch's gather (to_dev) or scatter into `list`;
// returns the number of chunks, or -1 when more than kMaxChunks are needed.
int chunk_list(const Slot& sl, dc_c64* dev, bool to_dev, CopyChunk* list) {
  int k = 0;
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    const Request* r = sl.reqs[i];
    for (long long o = 0; o < r->n; o += kCopyChunk) {
      if (k == kMaxChunks) return -1;
      const long long m = std::min<long long>(kCopyChunk, r->n - o);
      dc_c64* d = dev + sl.offs[i] + o;
      list[k++] = to_dev ? CopyChunk{r->x + o, d, m} : CopyChunk{d, r->y + o, m};
    }
  }
  return k;
}

// Hand a completed slot's results back (called with the lock held; drops it
// while copying: the slot's requests are in flight, which waiters and cancel
// leave alone).
void finish_slot(dc_server* s, Slot& sl, std::unique_lock<std::mutex>& lk) {
  const cudaError_t e = cudaEventQuery(sl.done);
  lk.unlock();
  if (e == cudaSuccess && !sl.direct_batch) {   // direct batches wrote the callers' buffers already
    std::vector<CopyPool::Job> jobs;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      jobs.push_back({sl.reqs[i]->y, sl.out_host + sl.offs[i], (size_t)sl.reqs[i]->n * sizeof(dc_c64)});
    s->copies->run(jobs);
  }
  const auto now = Clock::now();
  lk.lock();
  for (Request* r : sl.reqs) {
    r->state = e == cudaSuccess ? 2 : 3;
    r->status = e == cudaSuccess ? DC_OK : DC_ECUDA;
    if (e == cudaSuccess) s->done_samples += r->n;
    r->t_done = now;
    s->latencies.push_back(std::chrono::duration<double>(now - r->t_submit).count());
    ++s->completed;
  }
  s->t_last = now;
  s->alloc.release(sl.block, sl.block_bytes);
  sl.reqs.clear();
  sl.offs.clear();
  sl.busy = false;
  s->cv_done.notify_all();
}

// Device bytes of a batch: input and output (`samples`, 16-byte aligned
// offsets) and correct_batch's scratch for its items.
size_t batch_bytes(Slot& sl, const std::vector<dc_item>& items, long long samples,
                   size_t* scratch) {
  *scratch = dc_internal_batch_scratch(sl.ctx, items.data(), (int)items.size());
  return 2 * PoolAlloc::round((size_t)samples * sizeof(dc_c64)) + *scratch;
}

// Admit queued requests into a free slot and enqueue its work (called with
// the lock held; drops it while staging and enqueuing).  Requests join in
// arrival order while they fit the slot's staging and the pool can hold the
// whole batch (inputs, outputs, scratch); if even the first cannot be held,
// it waits for in-flight batches to return memory.
bool launch_slot(dc_server* s, Slot& sl, std::unique_lock<std::mutex>& lk) {
  long long used = 0;
  std::vector<dc_item> items;
  size_t bytes = 0, scratch = 0;
  while (!s->queue.empty()) {
    Request* r = s->queue.front();
    const long long need = (r->n + 1) & ~1LL;   // keep 16-byte alignment of offsets
    if (used + need > sl.cap) break;
    items.push_back(dc_item{used, r->n, used, r->n, r->fs, r->fc, r->v_r, r->tec});
    size_t sc = 0;
    const size_t b = batch_bytes(sl, items, used + need, &sc);
    if (PoolAlloc::round(b) > s->alloc.largest()) {   // the HBM budget is the limit now
      items.pop_back();
      if (items.empty() && !r->waited_memory) {
        r->waited_memory = true;
        ++s->waited_memory;
      }
      break;
    }
    bytes = b;
    scratch = sc;
    s->queue.pop_front();
    sl.reqs.push_back(r);
    sl.offs.push_back(used);
    used += need;
    r->state = 1;
  }
  if (sl.reqs.empty()) return false;
  if (!s->alloc.alloc(bytes, &sl.block)) {      // cannot happen: bytes <= largest free block
    for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) {
      (*it)->state = 0;
      s->queue.push_front(*it);
    }
    sl.reqs.clear();
    sl.offs.clear();
    return false;
  }
  sl.block_bytes = bytes;
  sl.busy = true;
  lk.unlock();
  char* base = s->pool + sl.block;
  const size_t io = PoolAlloc::round((size_t)used * sizeof(dc_c64));
  dc_c64* in_dev = reinterpret_cast<dc_c64*>(base);
  dc_c64* out_dev = reinterpret_cast<dc_c64*>(base + io);
  dc_status st = DC_OK;
  // direct: the gather and scatter lists (the slot's previous batch has
  // completed, so its lists are free)
  int n_in = -1, n_out = -1;
  if (s->direct) {
    n_in = chunk_list(sl, in_dev, true, sl.chunks);
    if (n_in >= 0) n_out = chunk_list(sl, out_dev, false, sl.chunks + kMaxChunks);
  }
  sl.direct_batch = n_in >= 0 && n_out >= 0;
  if (sl.direct_batch) {
    if (n_in > 0) copy_chunks_kernel<<<n_in, 256, 0, sl.stream>>>(sl.chunks);
    if (cudaGetLastError() != cudaSuccess) st = DC_ECUDA;
  } else {
    std::vector<CopyPool::Job> jobs;
    for (size_t i = 0; i < sl.reqs.size(); ++i)
      jobs.push_back({sl.in_host + sl.offs[i], sl.reqs[i]->x, (size_t)sl.reqs[i]->n * sizeof(dc_c64)});
    s->copies->run(jobs);
    if (cudaMemcpyAsync(in_dev, sl.in_host, (size_t)used * sizeof(dc_c64), cudaMemcpyHostToDevice,
                        sl.stream) != cudaSuccess)
      st = DC_ECUDA;
  }
  if (!st)
    st = dc_internal_correct_batch_ws(sl.ctx, in_dev, out_dev, items.data(), (int)items.size(),
                                      &s->opts, sl.stream, base + 2 * io, scratch);
  if (!st && sl.direct_batch) {
    if (n_out > 0) copy_chunks_kernel<<<n_out, 256, 0, sl.stream>>>(sl.chunks + kMaxChunks);
    if (cudaGetLastError() != cudaSuccess) st = DC_ECUDA;
  } else if (!st && cudaMemcpyAsync(sl.out_host, out_dev, (size_t)used * sizeof(dc_c64),
                                    cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess) {
    st = DC_ECUDA;
  }
  if (!st && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = DC_ECUDA;
  lk.lock();
  if (st) {
    const auto now = Clock::now();
    for (Request* r : sl.reqs) {
      r->state = 3;
      r->status = st;
      r->t_done = now;
    }
    if (cudaStreamSynchronize(sl.stream) == cudaSuccess) s->alloc.release(sl.block, sl.block_bytes);
    sl.reqs.clear();
    sl.offs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
    return false;
  }
  ++s->batches;
  return true;
}

void scheduler(dc_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    for (Slot& sl : s->slots)
      if (sl.busy && !sl.reqs.empty() && cudaEventQuery(sl.done) != cudaErrorNotReady) {
        finish_slot(s, sl, lk);
        progress = true;
      }
    bool any_free = false;
    for (Slot& sl : s->slots)
      if (!sl.busy && !s->queue.empty()) progress |= launch_slot(s, sl, lk);
    bool any_busy = false;
    for (Slot& sl : s->slots) {
      any_busy |= sl.busy;
      any_free |= !sl.busy;
    }
    if (!any_free && !s->queue.empty() && !s->queue.front()->waited_slot) {
      s->queue.front()->waited_slot = true;     // every slot busy: waits for a slot
      ++s->waited_slot;
    }
    if (s->stop && !any_busy) break;
    if (!progress) {
      // nothing to do right now: sleep until a submission, or poll the GPU
      if (any_busy || s->stop)
        s->cv_work.wait_for(lk, std::chrono::microseconds(50));
      else
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" dc_status dc_serve_start(int device, size_t hbm_budget_bytes, int slots, const dc_opts* opts,
                                    dc_server** out) {
  if (!out || slots < 1 || slots > 16) return DC_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return DC_EINVAL;
  dc_server* s = new dc_server();
  s->device = device;
  dc_opts_default(&s->opts);
  if (opts) s->opts = *opts;
  // The budget holds one device pool for the batches in flight (inputs,
  // outputs, correct_batch scratch) less a fixed reserve per slot for its
  // context's tables and item lists.  The pool must hold one 2^20-sample
  // request alone: 16 MiB in and out, 8 MiB resampled, 8 MiB four-step.
  constexpr long long kSlotMax = 32LL << 20;
  constexpr size_t kSlotReserve = (size_t)1 << 20;
  constexpr size_t kMinPool = ((size_t)32 << 20) + ((size_t)1 << 16);
  const size_t budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)8 << 30);
  if (budget < (size_t)slots * kSlotReserve + kMinPool) {
    delete s;
    return DC_EINVAL;            // the pool must hold the largest pulse (2^20 samples)
  }
  const size_t pool = (budget - (size_t)slots * kSlotReserve) & ~(size_t)255;
  s->cap = std::min<long long>((long long)(pool / (2 * sizeof(dc_c64))), kSlotMax);
  if (cudaMalloc(&s->pool, pool) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return DC_ENOMEM;
  }
  s->alloc.reset(pool);
  {
    // direct data movement where the device reaches pageable host memory
    // through the host's page tables
    int pageable = 0, host_tables = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
    cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device);
    const char* staged = getenv("DC_SERVE_STAGED");
    s->direct = pageable && host_tables && !(staged && staged[0] == '1');
    cudaGetLastError();
  }
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    sl.cap = s->cap;
    const size_t bytes = (size_t)sl.cap * sizeof(dc_c64);
    // the context's own scratch is never used (batches take theirs from the
    // pool), so its cap is one byte: any attempt to allocate fails loudly
    if (dc_create(&sl.ctx, device, 1) != DC_OK ||
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&sl.in_host, bytes) != cudaSuccess ||
        cudaMallocHost(&sl.out_host, bytes) != cudaSuccess ||
        cudaMallocHost(&sl.chunks, 2 * kMaxChunks * sizeof(CopyChunk)) != cudaSuccess) {
      cudaGetLastError();
      dc_serve_stop(s);
      return DC_ENOMEM;
    }
  }
  {
    const unsigned hw = std::thread::hardware_concurrency();
    s->copies = new CopyPool((int)std::max(1u, std::min(8u, hw > 2 ? hw - 2 : 1u)));
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return DC_OK;
}

extern "C" dc_status dc_serve_submit(dc_server* s, const dc_c64* x_host, long long n, double fs,
                                     double fc, double v_r, double tec_tecu, dc_c64* y_host,
                                     long long* req_id) {
  if (!s || !x_host || !y_host || !req_id) return DC_EINVAL;
  if (n < 1 || n > (1LL << 20) || n > s->cap) return DC_EINVAL;
  if (!(fs > 0.0) || !(fc >= 0.0) || (fc != 0.0 && !(fc > fs / 2.0)) || !(v_r > -299792458.0) ||
      !(v_r < 299792458.0) || !(tec_tecu == tec_tecu))
    return DC_EINVAL;
  Request* r = new Request{0, x_host, y_host, n, fs, fc, v_r, tec_tecu, Clock::now(), {}, 0, DC_OK};
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) {
      delete r;
      return DC_ECANCELLED;
    }
    r->id = s->next_id++;
    if (!s->have_first) {
      s->t_first = r->t_submit;
      s->have_first = true;
    }
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *req_id = r->id;
  }
  s->cv_work.notify_one();
  return DC_OK;
}

extern "C" dc_status dc_serve_wait(dc_server* s, long long id, int timeout_ms, double* latency_s) {
  if (!s) return DC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return DC_EINVAL;
  Request* r = it->second;
  const auto pred = [r] { return r->state >= 2; };
  if (timeout_ms < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return DC_ETIMEOUT;
  const dc_status st = r->state == 4 ? DC_ECANCELLED : r->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  s->reqs.erase(it);
  delete r;
  return st;
}

extern "C" dc_status dc_serve_cancel(dc_server* s, long long id) {
  if (!s) return DC_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return DC_EINVAL;
  Request* r = it->second;
  if (r->state != 0) return DC_EBUSY;     // already admitted to the GPU
  s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  r->state = 4;
  r->t_done = Clock::now();
  s->cv_done.notify_all();
  return DC_OK;
}

extern "C" dc_status dc_serve_stats(dc_server* s, double* p50_s, double* p99_s, double* msamples_per_s,
                                    long long* completed) {
  if (!s) return DC_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  std::vector<double> l = s->latencies;
  auto pct = [&l](double q) {
    if (l.empty()) return 0.0;
    const size_t k = std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5));
    std::nth_element(l.begin(), l.begin() + k, l.end());
    return l[k];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (msamples_per_s) {
    const double dt = s->have_first ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    *msamples_per_s = dt > 0 ? s->done_samples / dt / 1e6 : 0.0;
  }
  if (completed) *completed = s->completed;
  return DC_OK;
}

extern "C" dc_status dc_serve_stop(dc_server* s) {
  if (!s) return DC_EINVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  delete s->copies;
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) dc_destroy(sl.ctx);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.in_host) cudaFreeHost(sl.in_host);
    if (sl.out_host) cudaFreeHost(sl.out_host);
    if (sl.chunks) cudaFreeHost(sl.chunks);
  }
  if (s->pool) cudaFree(s->pool);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return DC_OK;
}

extern "C" dc_status dc_serve_counters(dc_server* s, dc_serve_info* out) {
  if (!s || !out) return DC_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  out->batches = s->batches;
  out->completed = s->completed;
  out->waited_memory = s->waited_memory;
  out->waited_slot = s->waited_slot;
  out->pool_bytes = s->alloc.total();
  out->peak_bytes_in_flight = s->alloc.peak();
  out->batch_capacity = s->cap;
  return DC_OK;
}
