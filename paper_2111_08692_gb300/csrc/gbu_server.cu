// gbu_server.cu -- the serving loop: continuous batching of validation and transcoding
// requests on one GPU (host code; the work runs in the library's kernels).
//
// A scheduler thread owns the device side.  Each pass it
//   1. retires launch groups whose completion event has fired: copies their results (already
//      in pinned host memory) into completion records, returns their input bytes to the
//      budget (outputs stay allocated until the caller releases them);
//   2. admits requests in submission order once their scheduled arrival time has passed,
//      while an in-flight slot is free and the device-memory budget (inputs + outputs of the
//      admitted requests) allows; each admitted transcoding gets its output buffer from the
//      server's device arena (worst-case size: n words for UTF-8 -> UTF-16LE, 3n bytes for
//      UTF-16LE -> UTF-8);
//   3. dispatches admitted requests into free launch-group slots: small requests of one
//      operation go together into ONE batched launch over device descriptors (warp per
//      string, CTA per longer string); requests of at least large_bytes each get a
//      single-buffer launch (all SMs on one string), several per group.  A group is: the
//      launches and an event.  Its descriptors and results either stay in mapped pinned host
//      memory, which the kernels read and write directly over the host link, or (device_rings)
//      live in device memory, with one copy of the descriptors before the launches and one
//      copy of the results after them.  Groups are spread round-robin over several streams,
//      so work admitted while earlier groups run overlaps with them on the device.
// Requests that arrive while the GPU is busy wait only for a free slot and memory, not for
// the earlier groups to finish: that is the continuous batching.  Latency = completion
// time (when the scheduler sees the event) - scheduled arrival time.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbu_device.cuh"
#include "gbu_internal.h"
#include "gbutf.h"

namespace {

uint64_t steady_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit offset allocator over [0, capacity) with coalescing of free neighbours.  Pure
// bookkeeping: it hands out offsets into a buffer that the owner allocated once.
class Arena {
 public:
  Arena(uint64_t capacity, uint64_t align) : cap_(capacity), align_(align ? align : 1), used_(0) {
    const uint64_t usable = capacity / align_ * align_;
    if (usable) free_[0] = usable;
  }
  bool alloc(uint64_t size, uint64_t *off) {
    if (size == 0) size = 1;
    size = (size + align_ - 1) / align_ * align_;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < size) continue;
      const uint64_t o = it->first, rest = it->second - size;
      free_.erase(it);
      if (rest) free_[o + size] = rest;
      live_[o] = size;
      used_ += size;
      *off = o;
      return true;
    }
    return false;
  }
  bool release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    uint64_t o = off, size = it->second;
    live_.erase(it);
    used_ -= size;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && o + size == nx->first) {  // merge with the next free block
      size += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {  // merge with the previous free block
      auto pv = std::prev(nx);
      if (pv->first + pv->second == o) {
        pv->second += size;
        return true;
      }
    }
    free_[o] = size;
    return true;
  }
  uint64_t used() const { return used_; }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto &f : free_) m = f.second > m ? f.second : m;
    return m;
  }
  uint64_t free_blocks() const { return free_.size(); }

 private:
  uint64_t cap_, align_, used_;
  std::map<uint64_t, uint64_t> free_;            // offset -> size
  std::unordered_map<uint64_t, uint64_t> live_;  // offset -> size
};

bool op_ok(int op) {
  return op == GBU_OP_VALIDATE_UTF8 || op == GBU_OP_VALIDATE_UTF16LE || op == GBU_OP_CONVERT_UTF8_TO_UTF16LE ||
         op == GBU_OP_CONVERT_UTF16LE_TO_UTF8;
}
uint64_t in_unit(int op) { return (op == GBU_OP_VALIDATE_UTF16LE || op == GBU_OP_CONVERT_UTF16LE_TO_UTF8) ? 2 : 1; }
// worst-case output bytes of a request (0 for validation)
uint64_t out_bytes(int op, uint64_t n) {
  if (op == GBU_OP_CONVERT_UTF8_TO_UTF16LE) return 2 * n;
  if (op == GBU_OP_CONVERT_UTF16LE_TO_UTF8) return 3 * n;
  return 0;
}
uint64_t out_cap(int op, uint64_t n) { return op == GBU_OP_CONVERT_UTF16LE_TO_UTF8 ? 3 * n : n; }
// output bytes charged to the budget (the arena's 256-byte granules)
uint64_t out_budget(int op, uint64_t n) {
  const uint64_t b = out_bytes(op, n);
  return b ? (b + 255) / 256 * 256 : 0;
}

struct Req {
  uint64_t id;
  gbu_request r;
  uint64_t admit_ns;
  uint64_t out_off;  // arena offset of the output (transcodings)
  bool cancelled;
};

struct Slot {
  cudaStream_t stream;
  cudaEvent_t done;
  gbu_ctx *ctx;
  gbu::StringDesc *desc_h;  // pinned, mapped
  gbu_result *res_h;        // pinned, mapped
  gbu::StringDesc *desc_d;  // what the kernels read: desc_h's device address, or a device copy
  gbu_result *res_d;        // what the kernels write: res_h's device address, or device memory
  uint32_t *pstart_h;       // pinned, mapped: first launch partition of each large request
  uint32_t *pstart_d;       // as desc_d
  void *rings_dev;          // device_rings: the device copies of desc, res and pstart (one allocation)
  gbu::SegState *seg_d;     // device: per-request error minimum / length / partitions done
  std::vector<Req> reqs;
  bool busy;
};

}  // namespace

struct gbu_server {
  int device;
  gbu_server_config cfg;
  uint64_t t0;  // server clock origin (steady clock ns)
  uint8_t *arena_base;
  Arena arena;
  std::vector<gbu_ctx *> ctxs;  // one per stream
  std::vector<cudaStream_t> streams;
  std::vector<Slot> slots;
  std::vector<std::deque<int>> issued;  // per stream: busy slots in issue order
  int next_stream;

  std::mutex mu;                       // guards everything below (and arena)
  std::deque<Req> pending;             // submitted, not admitted
  std::deque<gbu_completion> done;     // completed, not yet polled
  std::unordered_map<uint64_t, std::pair<uint64_t, uint64_t>> outputs;  // completed id -> (offset, bytes)
  uint64_t next_id;
  uint64_t budget_used;  // input bytes of admitted requests + arena bytes allocated
  uint64_t inflight;     // admitted, not completed
  gbu_server_stats stats;

  std::thread thread;
  std::atomic<bool> stop;

  gbu_server(uint64_t budget) : arena(budget, 256) {}
};

namespace {

uint64_t server_now(const gbu_server *s) { return steady_ns() - s->t0; }

void complete_locked(gbu_server *s, const Req &q, const gbu_result &res, uint64_t now) {
  gbu_completion c;
  memset(&c, 0, sizeof(c));
  c.id = q.id;
  c.tag = q.r.tag;
  c.result = res;
  c.dst = q.out_off != ~0ull ? (void *)(s->arena_base + q.out_off) : nullptr;
  c.arrival_ns = q.r.arrival_ns;
  c.admit_ns = q.admit_ns;
  c.complete_ns = now;
  if (q.out_off != ~0ull) {
    if (q.r.flags & GBU_REQ_DISCARD_OUTPUT) {
      s->arena.release(q.out_off);
      s->budget_used -= out_budget(q.r.op, q.r.n);
      c.dst = nullptr;
    } else {
      s->outputs[q.id] = {q.out_off, out_budget(q.r.op, q.r.n)};
    }
  }
  s->done.push_back(c);
  s->stats.completed++;
}

// Step 1: retire finished groups.  Groups on one stream finish in issue order, so only the
// oldest busy group of each stream is queried (one event query per stream per pass).
bool retire(gbu_server *s) {
  bool any = false;
  for (std::deque<int> &q_issued : s->issued) {
    while (!q_issued.empty()) {
      Slot &sl = s->slots[q_issued.front()];
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) break;
      const uint64_t now = server_now(s);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t k = 0; k < sl.reqs.size(); ++k) {
          const Req &q = sl.reqs[k];
          gbu_result r = sl.res_h[k];
          if (e != cudaSuccess) r = gbu_result{GBU_CUDA_ERROR, 0, 0};
          s->budget_used -= q.r.n * in_unit(q.r.op);
          s->inflight--;
          complete_locked(s, q, r, now);
        }
      }
      if (e != cudaSuccess) cudaGetLastError();
      sl.reqs.clear();
      sl.busy = false;
      q_issued.pop_front();
      any = true;
    }
  }
  return any;
}

// Step 2: admit arrived requests while slots and budget allow.
bool admit(gbu_server *s, std::deque<Req> &small_q, std::deque<Req> &large_q) {
  bool any = false;
  const uint64_t now = server_now(s);
  std::lock_guard<std::mutex> lk(s->mu);
  while (!s->pending.empty()) {
    Req &q = s->pending.front();
    if (q.cancelled) {
      complete_locked(s, q, gbu_result{GBU_CANCELLED, 0, 0}, now);
      s->pending.pop_front();
      any = true;
      continue;
    }
    if (q.r.arrival_ns > now) break;
    if (s->inflight >= s->cfg.max_inflight) break;
    const uint64_t ib = q.r.n * in_unit(q.r.op), ob = out_budget(q.r.op, q.r.n);
    if (s->budget_used + ib + ob > s->cfg.budget_bytes) break;
    q.out_off = ~0ull;
    if (ob) {
      uint64_t off;
      if (!s->arena.alloc(ob, &off)) break;  // fragmented: wait for releases
      q.out_off = off;
    }
    s->budget_used += ib + ob;
    s->inflight++;
    q.admit_ns = now;
    s->stats.admitted++;
    const uint64_t peak = s->budget_used;
    if (peak > s->stats.peak_budget_bytes) s->stats.peak_budget_bytes = peak;
    if (ib >= s->cfg.large_bytes) large_q.push_back(q);
    else small_q.push_back(q);
    s->pending.pop_front();
    any = true;
  }
  return any;
}

Slot *free_slot(gbu_server *s) {
  const int ns = (int)s->streams.size();
  const int per = s->cfg.groups_per_stream;
  for (int t = 0; t < ns; ++t) {
    const int st = (s->next_stream + t) % ns;
    for (int g = 0; g < per; ++g) {
      Slot &sl = s->slots[st * per + g];
      if (!sl.busy) {
        s->next_stream = (st + 1) % ns;
        return &sl;
      }
    }
  }
  return nullptr;
}

// Device rings: copies a group's B descriptors (and B + 1 partition starts) from the pinned
// staging into the slot's device memory on its stream, ahead of the launch that reads them.
int copy_descriptors(gbu_server *s, Slot &sl, size_t B, bool pstart) {
  if (!s->cfg.device_rings) return GBU_OK;
  if (cudaMemcpyAsync(sl.desc_d, sl.desc_h, B * sizeof(gbu::StringDesc), cudaMemcpyHostToDevice, sl.stream) !=
          cudaSuccess ||
      (pstart && cudaMemcpyAsync(sl.pstart_d, sl.pstart_h, (B + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                 sl.stream) != cudaSuccess))
    return GBU_CUDA_ERROR;
  return GBU_OK;
}

// Enqueues the group in sl (descriptors or single-buffer launches already decided).
void launch_group(gbu_server *s, Slot &sl, bool large) {
  const size_t B = sl.reqs.size();
  int rc = GBU_OK;
  const int op0 = sl.reqs[0].r.op;
  if (large && (op0 == GBU_OP_CONVERT_UTF8_TO_UTF16LE || op0 == GBU_OP_CONVERT_UTF16LE_TO_UTF8)) {
    // large transcodings of one direction: one launch over all their partitions, each
    // request with its own look-back chain
    uint32_t ntiles = 0;
    for (size_t k = 0; k < B; ++k) {
      const Req &q = sl.reqs[k];
      sl.desc_h[k].src = q.r.src;
      sl.desc_h[k].n = q.r.n;
      sl.desc_h[k].dst = (void *)(s->arena_base + q.out_off);
      sl.desc_h[k].cap = out_cap(op0, q.r.n);
      sl.pstart_h[k] = ntiles;
      ntiles += (uint32_t)gbu_internal_partitions(op0, q.r.src, q.r.n);
    }
    sl.pstart_h[B] = ntiles;
    rc = copy_descriptors(s, sl, B, true);
    if (rc == GBU_OK)
      rc = gbu_internal_convert_segments(sl.ctx, op0, sl.desc_d, sl.pstart_d, (uint32_t)B, ntiles, sl.seg_d, sl.res_d,
                                       sl.stream);
    s->stats.launches++;
  } else if (large) {
    for (size_t k = 0; k < B && rc == GBU_OK; ++k) {
      const Req &q = sl.reqs[k];
      const int op = q.r.op;
      uint8_t *dst = q.out_off != ~0ull ? s->arena_base + q.out_off : nullptr;
      gbu_result *res = sl.res_d + k;
      if (op == GBU_OP_VALIDATE_UTF8)
        rc = gbu_validate_utf8(sl.ctx, (const uint8_t *)q.r.src, q.r.n, res, sl.stream);
      else if (op == GBU_OP_VALIDATE_UTF16LE)
        rc = gbu_validate_utf16le(sl.ctx, (const uint16_t *)q.r.src, q.r.n, res, sl.stream);
      else if (op == GBU_OP_CONVERT_UTF8_TO_UTF16LE)
        rc = gbu_convert_utf8_to_utf16le(sl.ctx, (const uint8_t *)q.r.src, q.r.n, (uint16_t *)dst,
                                         out_cap(op, q.r.n), res, sl.stream);
      else
        rc = gbu_convert_utf16le_to_utf8(sl.ctx, (const uint16_t *)q.r.src, q.r.n, dst, out_cap(op, q.r.n), res,
                                         sl.stream);
      s->stats.launches++;
    }
  } else {
    const int op = sl.reqs[0].r.op;
    for (size_t k = 0; k < B; ++k) {
      const Req &q = sl.reqs[k];
      sl.desc_h[k].src = q.r.src;
      sl.desc_h[k].n = q.r.n;
      sl.desc_h[k].dst = q.out_off != ~0ull ? (void *)(s->arena_base + q.out_off) : nullptr;
      sl.desc_h[k].cap = out_bytes(op, q.r.n) ? out_cap(op, q.r.n) : 0;
    }
    // with host rings the kernel reads the descriptors and writes the results in mapped
    // pinned host memory, so a group costs its launches and one event, no copies
    rc = copy_descriptors(s, sl, B, false);
    if (rc == GBU_OK) rc = gbu_internal_batch_desc(sl.ctx, op, sl.desc_d, B, sl.res_d, sl.stream);
    s->stats.launches++;
  }
  if (rc == GBU_OK && s->cfg.device_rings &&
      cudaMemcpyAsync(sl.res_h, sl.res_d, B * sizeof(gbu_result), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
    rc = GBU_CUDA_ERROR;
  if (rc != GBU_OK) {
    // results of a group that could not be enqueued: report the failure, keep the slot usable
    cudaGetLastError();
    for (size_t k = 0; k < B; ++k) sl.res_h[k] = gbu_result{rc, 0, 0};
  }
  cudaEventRecord(sl.done, sl.stream);
  sl.busy = true;
  s->issued[(&sl - s->slots.data()) / s->cfg.groups_per_stream].push_back((int)(&sl - s->slots.data()));
  s->stats.groups++;
}

// Step 3: fill free slots.  Large requests first (oldest first); small ones of the operation
// whose oldest admitted request is oldest.
bool dispatch(gbu_server *s, std::deque<Req> &small_q, std::deque<Req> &large_q) {
  bool any = false;
  while (!small_q.empty() || !large_q.empty()) {
    Slot *sl = free_slot(s);
    if (!sl) break;
    if (!large_q.empty()) {
      // transcodings of the head's direction share one launch; validations run two per group
      const int op = large_q.front().r.op;
      const bool conv = op == GBU_OP_CONVERT_UTF8_TO_UTF16LE || op == GBU_OP_CONVERT_UTF16LE_TO_UTF8;
      const uint32_t lim = conv ? s->cfg.max_large_group : 2u;
      for (auto it = large_q.begin(); it != large_q.end() && sl->reqs.size() < lim;) {
        if (it->r.op == op) {
          sl->reqs.push_back(*it);
          it = large_q.erase(it);
        } else {
          ++it;
        }
      }
      launch_group(s, *sl, true);
    } else {
      const int op = small_q.front().r.op;
      for (auto it = small_q.begin(); it != small_q.end() && sl->reqs.size() < s->cfg.max_group;) {
        if (it->r.op == op) {
          sl->reqs.push_back(*it);
          it = small_q.erase(it);
        } else {
          ++it;
        }
      }
      launch_group(s, *sl, false);
    }
    any = true;
  }
  return any;
}

void run(gbu_server *s) {
  cudaSetDevice(s->device);
  std::deque<Req> small_q, large_q;  // admitted, not dispatched
  while (true) {
    bool any = retire(s);
    any |= admit(s, small_q, large_q);
    any |= dispatch(s, small_q, large_q);
    if (s->stop.load()) {
      bool busy = !small_q.empty() || !large_q.empty();
      for (const Slot &sl : s->slots) busy |= sl.busy;
      if (!busy) break;
    }
    if (!any) std::this_thread::yield();
  }
}

void destroy_resources(gbu_server *s) {
  for (Slot &sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.desc_h) cudaFreeHost(sl.desc_h);
    if (sl.res_h) cudaFreeHost(sl.res_h);
    if (sl.pstart_h) cudaFreeHost(sl.pstart_h);
    if (sl.seg_d) cudaFree(sl.seg_d);
    if (sl.rings_dev) cudaFree(sl.rings_dev);
  }
  for (gbu_ctx *c : s->ctxs) gbu_destroy(c);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->arena_base) cudaFree(s->arena_base);
}

}  // namespace

extern "C" void gbu_server_default_config(gbu_server_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->budget_bytes = 8ull << 30;
  // 16 streams x 8 groups in flight; large transcodings of one direction share a launch (up
  // to 32 requests), large validations run two per group
  cfg->streams = 16;
  cfg->groups_per_stream = 8;
  cfg->max_group = 4096;
  cfg->max_large_group = 32;
  cfg->large_bytes = 64 << 10;
  cfg->max_request_units = 16ull << 20;
  cfg->max_inflight = 1u << 16;
}

extern "C" gbu_server *gbu_server_create(int device, const gbu_server_config *cfg_in) {
  gbu_server_config cfg;
  gbu_server_default_config(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.streams < 1 || cfg.streams > 64 || cfg.groups_per_stream < 1 || cfg.groups_per_stream > 64 ||
      cfg.max_group < 1 || cfg.max_large_group < 1 || cfg.budget_bytes < 4096 || cfg.max_inflight < 1 ||
      cfg.max_request_units < 1)
    return nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return nullptr;
  gbu_server *s = new gbu_server(cfg.budget_bytes);
  s->device = device;
  s->cfg = cfg;
  s->arena_base = nullptr;
  s->next_stream = 0;
  s->next_id = 1;
  s->budget_used = 0;
  s->inflight = 0;
  memset(&s->stats, 0, sizeof(s->stats));
  s->stop = false;
  bool ok = cudaMalloc(&s->arena_base, cfg.budget_bytes) == cudaSuccess;
  for (int i = 0; ok && i < cfg.streams; ++i) {
    cudaStream_t st;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) break;
    s->streams.push_back(st);
    // look-back states for a whole group of large requests (max_large_group x the largest)
    gbu_ctx *c = gbu_create(device, (uint64_t)cfg.max_large_group * (cfg.max_request_units + 2 * gbu::PART_BYTES));
    ok = c != nullptr;
    if (ok) s->ctxs.push_back(c);
  }
  const uint32_t G = cfg.max_group > cfg.max_large_group ? cfg.max_group : cfg.max_large_group;
  s->slots.resize(ok ? (size_t)cfg.streams * cfg.groups_per_stream : 0);
  s->issued.resize(ok ? (size_t)cfg.streams : 0);
  for (size_t i = 0; ok && i < s->slots.size(); ++i) {
    Slot &sl = s->slots[i];
    sl.done = nullptr;
    sl.desc_h = nullptr;
    sl.res_h = nullptr;
    sl.desc_d = nullptr;
    sl.res_d = nullptr;
    sl.pstart_h = nullptr;
    sl.pstart_d = nullptr;
    sl.seg_d = nullptr;
    sl.rings_dev = nullptr;
    sl.stream = s->streams[i / cfg.groups_per_stream];
    sl.ctx = s->ctxs[i / cfg.groups_per_stream];
    sl.busy = false;
    ok = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaHostAlloc(&sl.desc_h, G * sizeof(gbu::StringDesc), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostAlloc(&sl.res_h, G * sizeof(gbu_result), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer((void **)&sl.desc_d, sl.desc_h, 0) == cudaSuccess &&
         cudaHostGetDevicePointer((void **)&sl.res_d, sl.res_h, 0) == cudaSuccess &&
         cudaHostAlloc(&sl.pstart_h, (G + 1) * sizeof(uint32_t), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer((void **)&sl.pstart_d, sl.pstart_h, 0) == cudaSuccess &&
         cudaMalloc(&sl.seg_d, G * sizeof(gbu::SegState)) == cudaSuccess;
    if (ok && cfg.device_rings) {
      // descriptors, results and partition starts in device memory instead (16-byte aligned parts)
      const size_t dbytes = G * sizeof(gbu::StringDesc), rbytes = G * sizeof(gbu_result);
      ok = cudaMalloc(&sl.rings_dev, dbytes + rbytes + (G + 1) * sizeof(uint32_t)) == cudaSuccess;
      if (ok) {
        sl.desc_d = static_cast<gbu::StringDesc *>(sl.rings_dev);
        sl.res_d = reinterpret_cast<gbu_result *>(static_cast<uint8_t *>(sl.rings_dev) + dbytes);
        sl.pstart_d = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(sl.rings_dev) + dbytes + rbytes);
      }
    }
    if (ok) {  // per-request states start {no error, 0, 0}
      std::vector<gbu::SegState> init(G);
      for (auto &e : init) e = gbu::SegState{gbu::NO_ERROR, 0ull, 0u, 0u};
      ok = cudaMemcpy(sl.seg_d, init.data(), G * sizeof(gbu::SegState), cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    destroy_resources(s);
    delete s;
    if (prev >= 0) cudaSetDevice(prev);
    return nullptr;
  }
  s->t0 = steady_ns();
  s->thread = std::thread(run, s);
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

extern "C" void gbu_server_destroy(gbu_server *s) {
  if (!s) return;
  {
    // requests not admitted yet are dropped (completed as cancelled, never polled)
    std::lock_guard<std::mutex> lk(s->mu);
    for (Req &q : s->pending) q.cancelled = true;
  }
  s->stop = true;
  s->thread.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  destroy_resources(s);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

extern "C" uint64_t gbu_server_now_ns(const gbu_server *s) { return s ? server_now(s) : 0; }

extern "C" int gbu_server_submit(gbu_server *s, const gbu_request *reqs, uint64_t count, uint64_t *first_id) {
  if (!s || (count > 0 && !reqs)) return GBU_BAD_ARGUMENT;
  for (uint64_t i = 0; i < count; ++i) {
    const gbu_request &r = reqs[i];
    if (!op_ok(r.op) || (r.n > 0 && !r.src) || r.n > s->cfg.max_request_units) return GBU_BAD_ARGUMENT;
    if (in_unit(r.op) == 2 && ((uintptr_t)r.src & 1)) return GBU_BAD_ARGUMENT;
    const uint64_t need = r.n * in_unit(r.op) + out_budget(r.op, r.n);
    if (need > s->cfg.budget_bytes) return GBU_OVER_BUDGET;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (first_id) *first_id = s->next_id;
  for (uint64_t i = 0; i < count; ++i) {
    Req q;
    q.id = s->next_id++;
    q.r = reqs[i];
    q.admit_ns = 0;
    q.out_off = ~0ull;
    q.cancelled = false;
    s->pending.push_back(q);
  }
  s->stats.submitted += count;
  return GBU_OK;
}

extern "C" int gbu_server_cancel(gbu_server *s, uint64_t id) {
  if (!s) return GBU_BAD_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req &q : s->pending) {
    if (q.id == id && !q.cancelled) {
      q.cancelled = true;
      return GBU_OK;
    }
  }
  return GBU_BAD_ARGUMENT;  // unknown, already admitted, or already cancelled
}

extern "C" int gbu_server_poll(gbu_server *s, gbu_completion *out, int max) {
  if (!s || !out || max < 0) return -GBU_BAD_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

extern "C" int gbu_server_release(gbu_server *s, uint64_t id) {
  if (!s) return GBU_BAD_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->outputs.find(id);  // only completed requests are listed
  if (it == s->outputs.end()) return GBU_BAD_ARGUMENT;
  s->arena.release(it->second.first);
  s->budget_used -= it->second.second;
  s->outputs.erase(it);
  return GBU_OK;
}

extern "C" int gbu_server_copy_output(gbu_server *s, uint64_t id, void *host, uint64_t bytes) {
  if (!s || (bytes > 0 && !host)) return GBU_BAD_ARGUMENT;
  uint64_t off, cap;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->outputs.find(id);
    if (it == s->outputs.end()) return GBU_BAD_ARGUMENT;
    off = it->second.first;
    cap = it->second.second;
  }
  if (bytes > cap) return GBU_BAD_ARGUMENT;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  const cudaError_t e = cudaMemcpy(host, s->arena_base + off, bytes, cudaMemcpyDeviceToHost);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBU_CUDA_ERROR;
  }
  return GBU_OK;
}

extern "C" int gbu_server_get_stats(gbu_server *s, gbu_server_stats *out) {
  if (!s || !out) return GBU_BAD_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->budget_used_bytes = s->budget_used;
  out->inflight = s->inflight;
  out->pending = s->pending.size();
  return GBU_OK;
}

// ---- host-side arena bookkeeping, exported for tests ---------------------------------------

struct gbu_arena {
  Arena a;
  explicit gbu_arena(uint64_t cap, uint64_t align) : a(cap, align) {}
};

extern "C" gbu_arena *gbu_arena_create(uint64_t capacity, uint64_t align) {
  if (align == 0 || (align & (align - 1))) return nullptr;
  return new gbu_arena(capacity, align);
}
extern "C" int gbu_arena_alloc(gbu_arena *a, uint64_t size, uint64_t *off) {
  if (!a || !off) return GBU_BAD_ARGUMENT;
  return a->a.alloc(size, off) ? GBU_OK : GBU_OVER_BUDGET;
}
extern "C" int gbu_arena_free(gbu_arena *a, uint64_t off) {
  if (!a) return GBU_BAD_ARGUMENT;
  return a->a.release(off) ? GBU_OK : GBU_BAD_ARGUMENT;
}
extern "C" uint64_t gbu_arena_used(const gbu_arena *a) { return a ? a->a.used() : 0; }
extern "C" uint64_t gbu_arena_largest_free(const gbu_arena *a) { return a ? a->a.largest_free() : 0; }
extern "C" uint64_t gbu_arena_free_blocks(const gbu_arena *a) { return a ? a->a.free_blocks() : 0; }
extern "C" void gbu_arena_destroy(gbu_arena *a) { delete a; }
