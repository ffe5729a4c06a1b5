// Continuous-batching request server (host code): admission by a device-memory budget,
// batches of one kind launched on free stream slots through the batched entry points,
// completions by CUDA events. The rules are stated with the declarations in fsz.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#if defined(__linux__)
#include <sys/prctl.h>
#endif

#include "../../include/fsz.h"

static_assert(sizeof(fsz_server_config) == 40 && sizeof(fsz_request) == 88 &&
                  sizeof(fsz_completion) == 48 && sizeof(fsz_server_stats) == 72,
              "ABI struct sizes");

namespace {

constexpr uint32_t kMaxSlots = 16;
constexpr uint32_t kMaxBatch = 4096;

uint64_t now_ns() {
  return uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(
                      std::chrono::steady_clock::now().time_since_epoch())
                      .count());
}

uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

uint64_t request_elems(const fsz_request& r) {
  if (r.kind == FSZ_REQ_DECOMPRESS) return r.n;
  uint64_t n = 1;
  for (uint32_t k = 0; k < r.dims.ndim && k < 3; ++k) n *= r.dims.dims[k];
  return n;
}

// The output allocation of one request inside its batch's arena.
uint64_t request_cap(const fsz_request& r) {
  if (r.kind == FSZ_REQ_COMPRESS) return align16(fsz_compress_bound(request_elems(r)));
  return align16(4 * std::max<uint64_t>(r.n, 4));
}

struct Req {
  fsz_request r;
  uint64_t cost;
  uint64_t arrival;
};

// One batch's output memory; freed when every output in it has been released.
struct Arena {
  void* base = nullptr;
  uint32_t refs = 0;
};

struct Held {
  Arena* arena;
  uint64_t cost;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* ws = nullptr;
  uint64_t ws_bytes = 0;
  void* h_table = nullptr;  // pinned: the batch's field descriptors
  void* d_table = nullptr;
  uint64_t* d_sizes = nullptr;
  uint64_t* h_sizes = nullptr;  // pinned
  std::vector<uint32_t> h_status;
  // the running batch
  bool busy = false;
  uint32_t kind = 0;
  std::vector<Req> batch;
  std::vector<uint64_t> offs;
  Arena* arena = nullptr;
  fsz_status code = FSZ_OK;
  uint64_t seq = 0;       // launch index of the running batch
  uint64_t deadline = 0;  // test mode
};

}  // namespace

struct fsz_server_s {
  fsz_server_config cfg{};
  bool sim = false;
  cudaMemPool_t pool = nullptr;
  std::vector<Slot> slots;

  std::mutex mu;                 // guards everything below
  std::condition_variable wake;  // the scheduler: arrivals, releases, stop
  std::condition_variable ready; // pollers: completions
  std::deque<Req> arrivals;
  std::deque<Req> pending;       // scheduler thread only
  std::deque<fsz_completion> completions;
  std::unordered_map<uint64_t, Held> held;
  uint64_t budget_free = 0;
  uint32_t inflight = 0;
  bool stop = false;
  fsz_server_stats st{};
  std::thread thread;

  void run();
  bool complete();
  bool launch();
  void finish(Slot& sl);
  fsz_status start_batch(Slot& sl, uint32_t kind, std::vector<Req>&& batch);
  void free_arena(Arena* a, cudaStream_t stream);
};

namespace {

fsz_status make_slot(Slot& sl, const fsz_server_config& c, cudaMemPool_t) {
  if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return FSZ_ERR_CUDA;
  if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) return FSZ_ERR_CUDA;
  // decompress outputs round each request up to 4 elements (16 bytes): room for that
  sl.ws_bytes = fsz_batch_workspace_bytes(c.max_batch_elems + 8ull * c.max_batch, c.max_batch);
  if (cudaMalloc(&sl.ws, sl.ws_bytes) != cudaSuccess) return FSZ_ERR_CUDA;
  const size_t tb = size_t(c.max_batch) * std::max(sizeof(fsz_cfield), sizeof(fsz_dfield));
  if (cudaMallocHost(&sl.h_table, tb) != cudaSuccess) return FSZ_ERR_CUDA;
  if (cudaMalloc(&sl.d_table, tb) != cudaSuccess) return FSZ_ERR_CUDA;
  if (cudaMalloc(&sl.d_sizes, 8 * size_t(c.max_batch)) != cudaSuccess) return FSZ_ERR_CUDA;
  if (cudaMallocHost(reinterpret_cast<void**>(&sl.h_sizes), 8 * size_t(c.max_batch)) != cudaSuccess)
    return FSZ_ERR_CUDA;
  sl.h_status.resize(c.max_batch);
  return FSZ_OK;
}

void free_slot(Slot& sl) {
  if (sl.stream) cudaStreamSynchronize(sl.stream);
  if (sl.ws) cudaFree(sl.ws);
  if (sl.d_table) cudaFree(sl.d_table);
  if (sl.d_sizes) cudaFree(sl.d_sizes);
  if (sl.h_table) cudaFreeHost(sl.h_table);
  if (sl.h_sizes) cudaFreeHost(sl.h_sizes);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.stream) cudaStreamDestroy(sl.stream);
}

}  // namespace

void fsz_server_s::free_arena(Arena* a, cudaStream_t stream) {
  if (a->base && !sim) cudaFreeAsync(a->base, stream);
  delete a;
}

fsz_status fsz_server_s::start_batch(Slot& sl, uint32_t kind, std::vector<Req>&& batch) {
  const uint32_t k = uint32_t(batch.size());
  sl.kind = kind;
  sl.batch = std::move(batch);
  sl.offs.assign(k, 0);
  uint64_t total = 0, n_total = 0;
  for (uint32_t i = 0; i < k; ++i) {
    sl.offs[i] = total;
    total += request_cap(sl.batch[i].r);
    n_total += request_elems(sl.batch[i].r);
  }
  sl.arena = new Arena();
  sl.arena->refs = k;
  sl.code = FSZ_OK;
  sl.busy = true;
  if (sim) {
    sl.deadline = now_ns() + cfg.sim_service_ns;
    return FSZ_OK;
  }
  if (cudaMallocFromPoolAsync(&sl.arena->base, total, pool, sl.stream) != cudaSuccess) {
    sl.code = FSZ_ERR_CUDA;
  } else if (kind == FSZ_REQ_COMPRESS) {
    auto* t = static_cast<fsz_cfield*>(sl.h_table);
    for (uint32_t i = 0; i < k; ++i) {
      const fsz_request& r = sl.batch[i].r;
      t[i].in = static_cast<const float*>(r.d_in);
      t[i].dims = r.dims;
      t[i].mode = fsz_eb_mode(r.mode);
      t[i].features_off = 0;
      t[i].eb = r.eb;
      t[i].out = static_cast<uint8_t*>(sl.arena->base) + sl.offs[i];
      t[i].out_capacity = request_cap(r);
      t[i].out_bytes = sl.d_sizes + i;
    }
    if (cudaMemcpyAsync(sl.d_table, sl.h_table, k * sizeof(fsz_cfield), cudaMemcpyHostToDevice,
                        sl.stream) != cudaSuccess) {
      sl.code = FSZ_ERR_CUDA;
    } else {
      sl.code = fsz_compress_batched(static_cast<const fsz_cfield*>(sl.d_table), k, n_total, sl.ws,
                                     sl.ws_bytes, reinterpret_cast<fsz_stream>(sl.stream));
      if (cudaMemcpyAsync(sl.h_sizes, sl.d_sizes, 8 * size_t(k), cudaMemcpyDeviceToHost, sl.stream) !=
          cudaSuccess)
        sl.code = FSZ_ERR_CUDA;
    }
  } else {
    auto* t = static_cast<fsz_dfield*>(sl.h_table);
    uint64_t cap_total = 0;
    for (uint32_t i = 0; i < k; ++i) {
      const fsz_request& r = sl.batch[i].r;
      t[i].in = r.d_in;
      t[i].in_bytes = r.in_bytes;
      t[i].out = reinterpret_cast<float*>(static_cast<uint8_t*>(sl.arena->base) + sl.offs[i]);
      t[i].out_capacity_elems = request_cap(r) / 4;
      cap_total += request_cap(r) / 4;
    }
    if (cudaMemcpyAsync(sl.d_table, sl.h_table, k * sizeof(fsz_dfield), cudaMemcpyHostToDevice,
                        sl.stream) != cudaSuccess) {
      sl.code = FSZ_ERR_CUDA;
    } else {
      sl.code = fsz_decompress_batched(static_cast<const fsz_dfield*>(sl.d_table), k, cap_total, sl.ws,
                                       sl.ws_bytes, reinterpret_cast<fsz_stream>(sl.stream));
    }
  }
  if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) sl.code = FSZ_ERR_CUDA;
  return sl.code;
}

// Turns a finished batch into completions; the outputs stay held until released.
void fsz_server_s::finish(Slot& sl) {
  const uint32_t k = uint32_t(sl.batch.size());
  fsz_status first = FSZ_OK;
  if (!sim && sl.code == FSZ_OK)
    first = fsz_check_batched(sl.ws, k, sl.h_status.data(), reinterpret_cast<fsz_stream>(sl.stream));
  const uint64_t t = now_ns();
  std::lock_guard<std::mutex> lk(mu);
  for (uint32_t i = 0; i < k; ++i) {
    const Req& q = sl.batch[i];
    fsz_completion c{};
    c.id = q.r.id;
    c.batch_size = k;
    c.batch = sl.seq;
    if (sim) {
      c.status = FSZ_OK;
    } else if (sl.code != FSZ_OK) {
      c.status = sl.code;
    } else {
      c.status = first == FSZ_ERR_CUDA ? FSZ_ERR_CUDA : int32_t(sl.h_status[i]);
    }
    c.d_out = sl.arena->base ? static_cast<uint8_t*>(sl.arena->base) + sl.offs[i] : nullptr;
    c.out_bytes = sim ? 0 : (q.r.kind == FSZ_REQ_COMPRESS ? sl.h_sizes[i] : 4 * q.r.n);
    c.latency_ns = t > q.arrival ? t - q.arrival : 0;
    held[q.r.id] = Held{sl.arena, q.cost};  // stays charged to the budget until released
    completions.push_back(c);
  }
  st.budget_free = budget_free;
  st.completed += k;
  sl.arena = nullptr;
  sl.batch.clear();
  sl.busy = false;
  --inflight;
  ready.notify_all();
}

bool fsz_server_s::complete() {
  bool any = false;
  for (Slot& sl : slots) {
    if (!sl.busy) continue;
    const bool done = sim ? now_ns() >= sl.deadline : cudaEventQuery(sl.done) != cudaErrorNotReady;
    if (done) {
      finish(sl);
      any = true;
    }
  }
  return any;
}

bool fsz_server_s::launch() {
  bool any = false;
  for (;;) {
    Slot* free_slot_ptr = nullptr;
    for (Slot& sl : slots)
      if (!sl.busy) {
        free_slot_ptr = &sl;
        break;
      }
    if (!free_slot_ptr || pending.empty()) return any;
    // Lingering: while batches run, a short batch waits for more requests for a while.
    if (cfg.linger_us > 0 && inflight > 0 && pending.size() < cfg.max_batch &&
        now_ns() < pending.front().arrival + uint64_t(cfg.linger_us) * 1000)
      return any;
    std::vector<Req> batch;
    uint32_t kind;
    {
      std::lock_guard<std::mutex> lk(mu);
      const Req& head = pending.front();
      if (head.cost > budget_free) return any;  // waits for released memory
      kind = head.r.kind;
      std::vector<Req> skipped;
      uint64_t reserved = 0, elems = 0;
      const uint32_t scan = cfg.scan ? cfg.scan : 4 * cfg.max_batch;
      for (uint32_t looked = 0; looked < scan && !pending.empty() && batch.size() < cfg.max_batch;
           ++looked) {
        Req q = pending.front();
        pending.pop_front();
        if (q.r.kind != kind) {  // waits for the next batch, its memory held back
          reserved += q.cost;
          skipped.push_back(q);
          continue;
        }
        const uint64_t e = request_elems(q.r);
        if (q.cost + reserved > budget_free || elems + e > cfg.max_batch_elems) {
          skipped.push_back(q);  // does not fit: nothing later overtakes it
          break;
        }
        budget_free -= q.cost;
        elems += e;
        batch.push_back(q);
      }
      for (auto it = skipped.rbegin(); it != skipped.rend(); ++it) pending.push_front(*it);
      if (inflight > 0) st.admitted_while_busy += batch.size();
      ++inflight;
      free_slot_ptr->seq = st.batches;
      st.batches += 1;
      st.max_inflight = std::max<uint64_t>(st.max_inflight, inflight);
      st.max_batch_seen = std::max<uint64_t>(st.max_batch_seen, batch.size());
      st.budget_free = budget_free;
      for (const Req& q : batch) st.bytes_in += 4 * request_elems(q.r);
    }
    start_batch(*free_slot_ptr, kind, std::move(batch));
    any = true;
  }
}

void fsz_server_s::run() {
#if defined(__linux__)
  // timed waits (event polling, lingering, future arrivals) to within a few microseconds
  // rather than the default 50 us timer slack
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
  for (;;) {
    bool stopping;
    {
      std::lock_guard<std::mutex> lk(mu);
      const uint64_t now = now_ns();
      while (!arrivals.empty()) {
        if (arrivals.front().arrival > now) break;  // submitted ahead of its arrival time
        Req q = arrivals.front();
        arrivals.pop_front();
        if (q.cost > cfg.budget_bytes || request_elems(q.r) > cfg.max_batch_elems) {
          fsz_completion c{};
          c.id = q.r.id;
          c.status = FSZ_ERR_REJECTED;
          c.batch = UINT64_MAX;
          const uint64_t t = now_ns();
          c.latency_ns = t > q.arrival ? t - q.arrival : 0;
          completions.push_back(c);
          st.rejected += 1;
          ready.notify_all();
          continue;
        }
        pending.push_back(q);
      }
      stopping = stop;
    }
    bool progressed = complete();
    progressed |= launch();
    if (stopping && inflight == 0 && !progressed && !pending.empty()) {
      // Stopping with requests that wait for memory the client still holds: nothing in
      // flight will return budget, so they are refused rather than waited for.
      std::lock_guard<std::mutex> lk(mu);
      const uint64_t t = now_ns();
      for (const Req& q : pending) {
        fsz_completion c{};
        c.id = q.r.id;
        c.status = FSZ_ERR_REJECTED;
        c.batch = UINT64_MAX;
        c.latency_ns = t > q.arrival ? t - q.arrival : 0;
        completions.push_back(c);
        st.rejected += 1;
      }
      pending.clear();
      ready.notify_all();
    }
    if (stopping && pending.empty() && inflight == 0) {
      std::lock_guard<std::mutex> lk(mu);
      if (arrivals.empty()) return;
    }
    if (!progressed) {
      // with batches on the GPU, poll their events every 20 us; otherwise sleep until
      // woken (a submission, a release, stop); never past the next held-back arrival
      std::unique_lock<std::mutex> lk(mu);
      uint64_t wait = inflight > 0 ? 20000 : 5000000;
      if (!arrivals.empty()) {
        const uint64_t now = now_ns(), a = arrivals.front().arrival;
        wait = std::min(wait, a > now ? a - now : 0);
      }
      if (wait > 0 && (inflight > 0 || !stop)) wake.wait_for(lk, std::chrono::nanoseconds(wait));
    }
  }
}

extern "C" {

uint64_t fsz_server_request_cost(const fsz_request* req) {
  if (req == nullptr) return 0;
  return request_cap(*req) + (req->kind == FSZ_REQ_COMPRESS ? 16 : 0);
}

fsz_status fsz_server_create(const fsz_server_config* cfg, fsz_server* out) {
  if (cfg == nullptr || out == nullptr) return FSZ_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > kMaxSlots || cfg->max_batch < 1 || cfg->max_batch > kMaxBatch ||
      cfg->linger_us > 10000000 || cfg->budget_bytes == 0 || cfg->max_batch_elems == 0)
    return FSZ_ERR_INVALID_ARG;
  auto* s = new fsz_server_s();
  s->cfg = *cfg;
  s->sim = cfg->sim_service_ns > 0;
  s->budget_free = cfg->budget_bytes;
  s->st.budget_free = cfg->budget_bytes;
  s->slots.resize(cfg->slots);
  if (!s->sim) {
    int dev = 0;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    fsz_status stat = FSZ_OK;
    if (cudaGetDevice(&dev) != cudaSuccess) stat = FSZ_ERR_CUDA;
    props.location.id = dev;
    if (stat == FSZ_OK && cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) stat = FSZ_ERR_CUDA;
    if (stat == FSZ_OK) {
      uint64_t keep = cfg->budget_bytes;  // keep freed arenas for reuse up to the budget
      cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (Slot& sl : s->slots)
      if (stat == FSZ_OK) stat = make_slot(sl, *cfg, s->pool);
    if (stat != FSZ_OK) {
      for (Slot& sl : s->slots) free_slot(sl);
      if (s->pool) cudaMemPoolDestroy(s->pool);
      delete s;
      return stat;
    }
  }
  s->thread = std::thread([s] { s->run(); });
  *out = s;
  return FSZ_OK;
}

static fsz_status check_request(const fsz_server_s* s, const fsz_request* req) {
  if (req->kind > FSZ_REQ_DECOMPRESS) return FSZ_ERR_INVALID_ARG;
  if (!s->sim && req->d_in == nullptr && request_elems(*req) > 0) return FSZ_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(req->d_in) & 15) return FSZ_ERR_ALIGN;
  return FSZ_OK;
}

fsz_status fsz_server_submit(fsz_server s, const fsz_request* req) {
  if (s == nullptr || req == nullptr) return FSZ_ERR_INVALID_ARG;
  return fsz_server_submit_many(s, req, 1);
}

fsz_status fsz_server_submit_many(fsz_server s, const fsz_request* h_reqs, uint64_t count) {
  if (s == nullptr || (h_reqs == nullptr && count > 0)) return FSZ_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < count; ++i) {
    const fsz_status e = check_request(s, &h_reqs[i]);
    if (e != FSZ_OK) return e;
  }
  const uint64_t now = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return FSZ_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < count; ++i) {
      Req q;
      q.r = h_reqs[i];
      q.cost = fsz_server_request_cost(&h_reqs[i]);
      q.arrival = h_reqs[i].arrival_ns ? h_reqs[i].arrival_ns : now;
      s->arrivals.push_back(q);
    }
    s->st.submitted += count;
  }
  s->wake.notify_one();
  return FSZ_OK;
}

uint32_t fsz_server_poll(fsz_server s, fsz_completion* h_out, uint32_t max, uint64_t wait_ns) {
  if (s == nullptr || h_out == nullptr || max == 0) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->completions.empty() && wait_ns > 0)
    s->ready.wait_for(lk, std::chrono::nanoseconds(wait_ns), [s] { return !s->completions.empty(); });
  uint32_t k = 0;
  while (k < max && !s->completions.empty()) {
    h_out[k++] = s->completions.front();
    s->completions.pop_front();
  }
  return k;
}

fsz_status fsz_server_release(fsz_server s, uint64_t id, fsz_stream stream) {
  return fsz_server_release_many(s, &id, 1, stream);
}

fsz_status fsz_server_release_many(fsz_server s, const uint64_t* h_ids, uint64_t count,
                                   fsz_stream stream) {
  if (s == nullptr || (h_ids == nullptr && count > 0)) return FSZ_ERR_INVALID_ARG;
  fsz_status code = FSZ_OK;
  std::vector<Arena*> to_free;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t i = 0; i < count; ++i) {
      auto it = s->held.find(h_ids[i]);
      if (it == s->held.end()) {
        code = FSZ_ERR_INVALID_ARG;
        continue;
      }
      if (--it->second.arena->refs == 0) to_free.push_back(it->second.arena);
      s->budget_free += it->second.cost;
      s->held.erase(it);
    }
    s->st.budget_free = s->budget_free;
  }
  for (Arena* a : to_free) s->free_arena(a, reinterpret_cast<cudaStream_t>(stream));
  s->wake.notify_one();  // memory returned: waiting requests may fit now
  return code;
}

fsz_status fsz_server_get_stats(fsz_server s, fsz_server_stats* h_stats) {
  if (s == nullptr || h_stats == nullptr) return FSZ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *h_stats = s->st;
  h_stats->budget_free = s->budget_free;
  return FSZ_OK;
}

fsz_status fsz_server_stop(fsz_server s) {
  if (s == nullptr) return FSZ_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->wake.notify_all();
  return FSZ_OK;
}

fsz_status fsz_server_destroy(fsz_server s) {
  if (s == nullptr) return FSZ_ERR_INVALID_ARG;
  fsz_server_stop(s);
  if (s->thread.joinable()) s->thread.join();
  std::vector<Arena*> arenas;
  for (auto& kv : s->held)
    if (std::find(arenas.begin(), arenas.end(), kv.second.arena) == arenas.end())
      arenas.push_back(kv.second.arena);
  for (Arena* a : arenas) s->free_arena(a, nullptr);
  if (!s->sim) {
    cudaDeviceSynchronize();
    for (Slot& sl : s->slots) free_slot(sl);
    if (s->pool) cudaMemPoolDestroy(s->pool);
  }
  delete s;
  return FSZ_OK;
}

fsz_status fsz_copy_device(void* d_dst, const void* d_src, uint64_t bytes, fsz_stream stream) {
  if (bytes == 0) return FSZ_OK;
  if (d_dst == nullptr || d_src == nullptr) return FSZ_ERR_INVALID_ARG;
  return cudaMemcpyAsync(d_dst, d_src, bytes, cudaMemcpyDeviceToDevice,
                         reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FSZ_OK
             : FSZ_ERR_CUDA;
}

}  // extern "C"
