// server.cu -- continuous batching of permute-scale-add requests
// (include/ttc.h, ttc_server_*).
//
// Threads: the caller submits; a scheduler thread admits pending requests in
// arrival order under the memory budget, groups them into an epoch and
// launches it on a lane (a stream with a ring of descriptor slots in pinned
// host and device memory); a completion thread queries the oldest epoch of
// each lane (a stream completes its work in order), stamps latencies and
// releases budget.  Several small requests of an epoch share the batched
// launches, one per class (batch_impl.h); a large request, or a small one that
// arrived alone, gets the single-plan kernel.  Lanes run concurrently, so new
// requests overlap on the device with work in flight, and the least-loaded
// lane takes the next epoch, so small requests need not queue behind a large
// one.  Requests fall into size classes with streams of their own, smaller
// classes at higher stream priority: the block scheduler then starts a small
// request's thread blocks ahead of the waiting blocks of a large one.
#include <cuda_runtime.h>
#include <sys/prctl.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "../../include/ttc.h"
#include "batch_impl.h"
#include "launch.h"
#include "plan_impl.h"
#include "planner.h"

using namespace ttc;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kSlotBytes = size_t(4) << 20;   // descriptors + tables + tile records of one batched epoch
constexpr int kSlots = 8;                        // batched epochs in flight per lane
constexpr int kLaneMaxQueued = 64;               // epochs in flight per lane
constexpr int kMaxEpoch = 1024;                  // requests per batched epoch
constexpr double kWatchdogS = 30.0;              // default: an epoch older than this is given up
constexpr int64_t kMediumBytes = int64_t(64) << 20;  // largest algorithmic bytes of size class 1
constexpr double kIdleSpinS = 50e-6;             // the scheduler polls this long before it sleeps

enum ReqState : int { RQ_PENDING = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Req {
  ttc_plan_t plan;
  const void* A;
  void* B;
  int64_t bytes;       // admission bytes (A and B spans)
  int64_t alg_bytes;   // algorithmic bytes
  int64_t tiles;       // tiles in the batch body, or -1 if it cannot take the request
  int cls;             // size class: 0 batchable, 1 medium, 2 large
  uint64_t delay_ns = 0;  // plan == nullptr: a bounded delay kernel (tests)
  double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
  int state = RQ_PENDING;
  ttc_status status = TTC_OK;
};

struct Epoch {
  cudaEvent_t ev;
  std::vector<int64_t> reqs;
  int64_t bytes;
  int slot;            // descriptor slot it holds, or -1
  double t_launch;
  std::vector<ttc_plan_t> fp8_plans;
};

struct Lane {
  cudaStream_t s = nullptr;
  int cls = 0;               // size class it serves
  char* d_slots = nullptr;   // kSlots x kSlotBytes
  char* h_slots = nullptr;
  int slot_next = 0, slots_used = 0;
  bool dead = false;         // an epoch on it was given up by the watchdog
  int64_t load = 0;          // bytes of its epochs in flight
  std::deque<Epoch> q;       // epochs in flight, in stream order
};

}  // namespace

struct ttc_server_s {
  double watchdog_s = kWatchdogS;
  int64_t budget = 0;
  int64_t small_tiles = 0;
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_poll;
  std::deque<Req> reqs;              // ticket = index (references stay valid)
  std::deque<int64_t> pending;
  std::atomic<int64_t> npending{0};  // pending.size(), readable without the lock
  std::atomic<bool> stop_flag{false};
  std::vector<Lane> lanes;
  std::vector<cudaEvent_t> free_events;
  std::set<ttc_plan_t> fp8_busy;
  int launching = 0;                 // epochs taken from `pending` but not yet on a lane
  int inflight = 0;                  // epochs on lanes
  int64_t inflight_bytes = 0, peak_inflight = 0;
  int64_t n_epochs = 0, n_launches = 0, n_completed = 0, n_failed = 0, done_bytes = 0;
  std::vector<double> latencies_us;
  double first_submit = 0, last_complete = 0;
  bool stop = false;
  std::thread sched, compl_thread;
};

namespace {

bool is_small(const ttc_server_s* S, const Req& r) { return r.tiles >= 0 && r.tiles <= S->small_tiles; }

// Lay out the batched launch of `small` in descriptor slot `slot` of lane L
// (pinned staging, then one copy to the device slot on the lane's stream)
// and launch it.  Per problem the host writes its descriptor, its offset
// tables and its first global tile; the kernel derives the tiles' records.
ttc_status launch_batched(Lane& L, int slot, const std::vector<Req*>& small, int* launches) {
  std::vector<BatchDesc> descs;
  std::vector<int32_t> tabs;
  std::vector<size_t> tab_at, tab_na;
  std::vector<uint32_t> tile0;
  int smem = 0;
  uint64_t total = 0;
  for (Req* r : small) {
    BatchDesc d;
    size_t na = 0;
    const size_t at = tabs.size();
    if (!batch_describe(r->plan, r->A, r->B, &d, &tabs, &na, &smem)) continue;
    descs.push_back(d);
    tab_at.push_back(at);
    tab_na.push_back(na);
  }
  // ordered by class (one kernel launch per class), then the first tiles
  {
    std::vector<size_t> idx(descs.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](size_t x, size_t y) { return batch_class(descs[x]) < batch_class(descs[y]); });
    std::vector<BatchDesc> d2;
    std::vector<size_t> at2, na2;
    for (size_t i : idx) {
      d2.push_back(descs[i]);
      at2.push_back(tab_at[i]);
      na2.push_back(tab_na[i]);
    }
    descs.swap(d2);
    tab_at.swap(at2);
    tab_na.swap(na2);
  }
  for (BatchDesc& d : descs) {
    d.tile0 = uint32_t(total);
    tile0.push_back(uint32_t(total));
    total += d.ntiles;
  }
  std::vector<BatchRange> ranges;
  batch_ranges(descs, &ranges);
  if (descs.empty()) return TTC_OK;
  const size_t off_tab = (descs.size() * sizeof(BatchDesc) + 255) & ~size_t(255);
  const size_t off_t0 = (off_tab + tabs.size() * 4 + 255) & ~size_t(255);
  const size_t off_cnt = (off_t0 + tile0.size() * 4 + 255) & ~size_t(255);   // end of the epoch's data
  if (off_cnt + 256 > kSlotBytes) return fail(TTC_ERR_INVALID_SIZE, "epoch exceeds the descriptor slot");
  char* hb = L.h_slots + size_t(slot) * kSlotBytes;
  char* db = L.d_slots + size_t(slot) * kSlotBytes;
  int32_t* d_tab = reinterpret_cast<int32_t*>(db + off_tab);
  for (size_t i = 0; i < descs.size(); ++i) {
    if (descs[i].path != BP_COPY) {
      descs[i].tp.tabA = d_tab + tab_at[i];
      descs[i].tp.tabB = d_tab + tab_at[i] + tab_na[i];
    }
  }
  std::memcpy(hb, descs.data(), descs.size() * sizeof(BatchDesc));
  if (!tabs.empty()) std::memcpy(hb + off_tab, tabs.data(), tabs.size() * 4);
  std::memcpy(hb + off_t0, tile0.data(), tile0.size() * 4);
  cudaError_t e = cudaMemcpyAsync(db, hb, off_cnt, cudaMemcpyHostToDevice, L.s);
  if (e != cudaSuccess) return cuda_fail(e, "server descriptor upload");
  e = batch_launch(reinterpret_cast<BatchDesc*>(db), nullptr, reinterpret_cast<uint32_t*>(db + off_t0),
                   uint32_t(descs.size()), ranges, smem, L.s);
  if (e != cudaSuccess) return cuda_fail(e, "server batch launch");
  *launches += int64_t(ranges.size());
  return TTC_OK;
}

// Fail every pending request (no lane can run work any more).
void fail_pending(ttc_server_s* S) {
  for (int64_t t : S->pending) {
    Req& r = S->reqs[size_t(t)];
    r.status = TTC_ERR_TIMEOUT;
    r.state = RQ_DONE;
    r.t_done = now_s();
    S->n_failed += 1;
  }
  S->pending.clear();
  S->npending.store(0, std::memory_order_release);
  S->cv_poll.notify_all();
}

void scheduler(ttc_server_s* S) {
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop && S->pending.empty()) break;
    if (S->pending.empty()) {
      // poll for a short while before sleeping: waking a sleeping thread
      // costs ~10 us, which every request arriving to an idle queue would wait
      lk.unlock();
      const double until = now_s() + kIdleSpinS;
      while (S->npending.load(std::memory_order_acquire) == 0 && !S->stop_flag.load() && now_s() < until)
        std::this_thread::yield();
      lk.lock();
      if (S->pending.empty() && !S->stop) S->cv_sched.wait(lk);
      continue;
    }
    if (std::all_of(S->lanes.begin(), S->lanes.end(), [](const Lane& L) { return L.dead; })) {
      fail_pending(S);
      continue;
    }
    // The front request decides the kind of epoch: a large request runs
    // alone (its budget is released as soon as it finishes), small ones are
    // gathered in arrival order into one batched launch.
    Req& front = S->reqs[size_t(S->pending.front())];
    const bool f_small = is_small(S, front);
    const int f_cls = front.cls;
    if (std::none_of(S->lanes.begin(), S->lanes.end(),
                     [&](const Lane& L) { return L.cls == f_cls && !L.dead; })) {
      // every stream of its size class was given up by the watchdog
      front.status = TTC_ERR_TIMEOUT;
      front.state = RQ_DONE;
      front.t_done = now_s();
      S->n_failed += 1;
      S->pending.pop_front();
      S->npending.store(int64_t(S->pending.size()), std::memory_order_release);
      S->cv_poll.notify_all();
      continue;
    }
    int lane = -1;
    for (int i = 0; i < int(S->lanes.size()); ++i) {
      const Lane& c = S->lanes[size_t(i)];
      if (c.cls != f_cls || c.dead || int(c.q.size()) >= kLaneMaxQueued || (f_small && c.slots_used == kSlots)) continue;
      if (lane < 0 || c.load < S->lanes[size_t(lane)].load) lane = i;
    }
    if (lane < 0) {
      S->cv_sched.wait(lk);
      continue;
    }
    // admission: arrival order, while the budget allows
    std::vector<int64_t> take;
    int64_t ebytes = 0;
    size_t slot_need = 4096;
    while (!S->pending.empty() && int(take.size()) < kMaxEpoch) {
      Req& r = S->reqs[size_t(S->pending.front())];
      if (S->inflight_bytes + ebytes + r.bytes > S->budget) break;
      const bool fp8 = r.plan && r.plan->dout == DT_E4M3;
      if (fp8 && S->fp8_busy.count(r.plan)) break;      // that plan's scale scratch is in use
      const bool small = is_small(S, r);
      if (small != f_small || r.cls != f_cls) break;
      if (small) {
        const size_t need = sizeof(BatchDesc) + 16384 + 4;
        if (slot_need + need > kSlotBytes) break;
        slot_need += need;
      }
      if (fp8) S->fp8_busy.insert(r.plan);
      take.push_back(S->pending.front());
      S->pending.pop_front();
      S->npending.store(int64_t(S->pending.size()), std::memory_order_release);
      ebytes += r.bytes;
      if (!small) break;
    }
    if (take.empty()) {
      S->cv_sched.wait(lk);
      continue;
    }
    Lane& L = S->lanes[size_t(lane)];
    // several small requests share a batched launch; one alone takes the
    // single-plan kernel, which is faster for a single problem
    const bool batched = f_small && take.size() > 1;
    int slot = -1;
    if (batched) {
      slot = L.slot_next;
      L.slot_next = (L.slot_next + 1) % kSlots;
      L.slots_used += 1;
    }
    S->inflight_bytes += ebytes;
    S->peak_inflight = std::max(S->peak_inflight, S->inflight_bytes);
    L.load += ebytes;
    // events come from the pool made at creation: a lane holds at most
    // kLaneMaxQueued epochs, so the pool never runs dry
    cudaEvent_t ev = S->free_events.back();
    S->free_events.pop_back();
    std::vector<Req*> rs;
    std::vector<ttc_plan_t> fp8s;
    const double ta = now_s();
    for (int64_t t : take) {
      Req& r = S->reqs[size_t(t)];
      r.state = RQ_RUNNING;
      r.t_admit = ta;
      if (r.plan && r.plan->dout == DT_E4M3) fp8s.push_back(r.plan);
      rs.push_back(&r);
    }
    S->launching += 1;
    lk.unlock();
    // launch outside the lock (only this thread touches L's slots and stream)
    ttc_status st = TTC_OK;
    int launches = 0;
    if (batched) {
      st = launch_batched(L, slot, rs, &launches);
    } else {
      for (Req* r : rs) {
        if (st != TTC_OK) break;
        if (r->plan) {
          st = run_plan(r->plan, r->A, r->B, L.s);
        } else {
          const cudaError_t de = launch_delay(r->delay_ns, L.s);
          st = de == cudaSuccess ? TTC_OK : cuda_fail(de, "delay kernel launch");
        }
        ++launches;
      }
    }
    cudaEventRecord(ev, L.s);
    const double tl = now_s();
    lk.lock();
    for (int64_t t : take) {
      S->reqs[size_t(t)].t_launch = tl;
      if (st != TTC_OK) S->reqs[size_t(t)].status = st;
    }
    L.q.push_back({ev, take, ebytes, slot, tl, fp8s});
    S->launching -= 1;
    S->inflight += 1;
    S->n_epochs += 1;
    S->n_launches += launches;
    S->cv_done.notify_all();
  }
}

// Finish the requests of epoch e of lane L (d: 1 done, 2 failed, 3 given up).
void retire(ttc_server_s* S, Lane& L, Epoch& e, int d, double t) {
  for (int64_t tk : e.reqs) {
    Req& r = S->reqs[size_t(tk)];
    if (d == 2 && r.status == TTC_OK) r.status = TTC_ERR_CUDA;
    if (d == 3 && r.status == TTC_OK) r.status = TTC_ERR_TIMEOUT;
    r.state = RQ_DONE;
    r.t_done = t;
    if (r.status == TTC_OK) {
      S->n_completed += 1;
      S->done_bytes += r.alg_bytes;
      S->latencies_us.push_back((t - r.t_submit) * 1e6);
      S->last_complete = std::max(S->last_complete, t);
    } else {
      S->n_failed += 1;
    }
  }
  for (ttc_plan_t p : e.fp8_plans) S->fp8_busy.erase(p);
  S->inflight_bytes -= e.bytes;
  S->inflight -= 1;
  L.load -= e.bytes;
  if (d == 3) {
    // given up: the stream may still be running it, so neither the lane
    // (its slots) nor the event is used again
    L.dead = true;
  } else {
    if (e.slot >= 0) L.slots_used -= 1;
    S->free_events.push_back(e.ev);
  }
}

void completer(ttc_server_s* S) {
  cudaSetDevice(S->dev);
  // short sleeps between polls must not be stretched by the default timer
  // slack (tens of microseconds), which would add to every latency
  prctl(PR_SET_TIMERSLACK, 1UL, 0, 0, 0);
  std::unique_lock<std::mutex> lk(S->mu);
  std::vector<std::pair<int, cudaEvent_t>> heads;
  std::vector<double> t_launch;
  std::vector<int> done;
  while (true) {
    if (S->inflight == 0) {
      if (S->stop && S->pending.empty() && S->launching == 0) break;
      S->cv_done.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    // The oldest epoch of each lane: a stream finishes its work in order,
    // so later epochs of a lane cannot be done before it.
    bool any = false;
    while (true) {
      heads.clear();
      t_launch.clear();
      for (int i = 0; i < int(S->lanes.size()); ++i) {
        const Lane& L = S->lanes[size_t(i)];
        if (!L.q.empty() && !L.dead) {
          heads.push_back({i, L.q.front().ev});
          t_launch.push_back(L.q.front().t_launch);
        }
      }
      if (heads.empty()) break;
      lk.unlock();
      done.assign(heads.size(), 0);
      const double t0 = now_s();
      for (size_t i = 0; i < heads.size(); ++i) {
        const cudaError_t q = cudaEventQuery(heads[i].second);
        if (q == cudaSuccess) done[i] = 1;
        else if (q != cudaErrorNotReady) done[i] = 2;           // the epoch failed
        else if (t0 - t_launch[i] > S->watchdog_s) done[i] = 3;  // watchdog
      }
      const double t = now_s();
      lk.lock();
      bool progressed = false;
      for (size_t i = 0; i < heads.size(); ++i) {
        if (!done[i]) continue;
        Lane& L = S->lanes[size_t(heads[i].first)];
        // only this thread removes epochs, so the head is still the same
        retire(S, L, L.q.front(), done[i], t);
        L.q.pop_front();
        if (L.dead) {
          // what was queued behind a given-up epoch is given up with it
          while (!L.q.empty()) {
            retire(S, L, L.q.front(), 3, t);
            L.q.pop_front();
          }
        }
        progressed = true;
      }
      if (!progressed) break;
      any = true;
    }
    if (any) {
      S->cv_sched.notify_all();
      S->cv_poll.notify_all();
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(2));
      lk.lock();
    }
  }
}

void free_lanes(std::vector<Lane>& lanes) {
  for (auto& L : lanes) {
    if (L.dead) {
      // its stream may still run a given-up epoch: waiting for it, or
      // freeing memory it may use (cudaFree synchronises), could block
      // forever, so the stream is released without a wait and its slots
      // are left allocated
      if (L.s) cudaStreamDestroy(L.s);
      L = Lane();
      continue;
    }
    if (L.s) {
      cudaStreamSynchronize(L.s);
      cudaStreamDestroy(L.s);
    }
    if (L.d_slots) cudaFree(L.d_slots);
    if (L.h_slots) cudaFreeHost(L.h_slots);
    L = Lane();
  }
}

}  // namespace

extern "C" {

ttc_status ttc_server_create(ttc_server_t* out, int64_t budget_bytes, int nstreams, int64_t small_tiles) {
  if (!out) return fail(TTC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (budget_bytes <= 0 || nstreams < 1 || nstreams > 16 || small_tiles < 0)
    return fail(TTC_ERR_INVALID_ARG, "bad server configuration");
  std::unique_ptr<ttc_server_s> S(new (std::nothrow) ttc_server_s());
  if (!S) return fail(TTC_ERR_OOM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&S->dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  S->budget = budget_bytes;
  S->small_tiles = small_tiles;
  // size classes: 0 batchable (highest priority), 1 medium, 2 large
  // (lowest); one class at default priority when batching is off
  const int nclass = small_tiles > 0 ? 3 : 1;
  int least = 0, greatest = 0;
  if (nclass > 1) {
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetStreamPriorityRange");
  }
  const int prio[3] = {greatest, (least + greatest) / 2, least};
  S->lanes.resize(size_t(nclass * nstreams));
  for (size_t i = 0; i < S->lanes.size(); ++i) {
    Lane& L = S->lanes[i];
    L.cls = int(i) / nstreams;
    e = nclass > 1 ? cudaStreamCreateWithPriority(&L.s, cudaStreamNonBlocking, prio[L.cls])
                   : cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
    if (e == cudaSuccess && small_tiles > 0 && L.cls == 0) e = cudaMalloc(&L.d_slots, kSlots * kSlotBytes);
    if (e == cudaSuccess && small_tiles > 0 && L.cls == 0) e = cudaMallocHost(&L.h_slots, kSlots * kSlotBytes);
    if (e != cudaSuccess) {
      free_lanes(S->lanes);
      return e == cudaErrorMemoryAllocation ? fail(TTC_ERR_OOM, "server allocation failed")
                                            : cuda_fail(e, "server setup");
    }
  }
  const size_t nev = S->lanes.size() * size_t(kLaneMaxQueued);
  for (size_t i = 0; i < nev; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (auto x : S->free_events) cudaEventDestroy(x);
      free_lanes(S->lanes);
      return cuda_fail(e, "server event creation");
    }
    S->free_events.push_back(ev);
  }
  S->sched = std::thread(scheduler, S.get());
  S->compl_thread = std::thread(completer, S.get());
  *out = S.release();
  return TTC_OK;
}

ttc_status ttc_server_submit(ttc_server_t S, ttc_plan_t plan, const void* A, void* B, int64_t* ticket) {
  if (!S || !plan || !ticket) return fail(TTC_ERR_INVALID_ARG, "NULL argument");
  Req r;
  r.plan = plan;
  r.A = A;
  r.B = B;
  const int sa = dtype_size(plan->din), sb = dtype_size(plan->dout);
  r.bytes = plan->canon.spanA * sa + plan->canon.spanB * sb;
  r.alg_bytes = plan->canon.n * (sa + (plan->beta_nonzero() ? 2 * sb : sb));
  if (r.bytes > S->budget) return fail(TTC_ERR_BUDGET, "request larger than the server's memory budget");
  if (plan->canon.n > 0) {
    if (!A || !B) return fail(TTC_ERR_INVALID_ARG, "A or B is NULL");
    const uintptr_t a = reinterpret_cast<uintptr_t>(A), b = reinterpret_cast<uintptr_t>(B);
    if (a % sa || b % sb) return fail(TTC_ERR_ALIGN, "A or B not aligned to its element size");
    if (a < b + uintptr_t(plan->canon.spanB) * sb && b < a + uintptr_t(plan->canon.spanA) * sa)
      return fail(TTC_ERR_ALIAS, "the byte ranges of A and B overlap");
  }
  r.tiles = -1;
  // FP8 (grid-wide amax) and complex requests are never batched
  if (S->small_tiles > 0 && plan->dout != DT_E4M3 && !is_complex(plan->din) && plan->canon.n > 0)
    r.tiles = batch_tiles(plan);
  if (plan->canon.n > 0) {
    // the plan's device scratch and tables are set up here, on the caller's
    // thread, the first time the plan meets this device: done by the
    // scheduler it would stall every request queued behind this one
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != S->dev) e = cudaSetDevice(S->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    DevRes* res = nullptr;
    const ttc_status st = ensure_device(plan, S->dev, &res);
    if (cur != S->dev) cudaSetDevice(cur);
    if (st != TTC_OK) return st;
  }
  r.cls = S->small_tiles == 0 ? 0 : is_small(S, r) ? 0 : r.alg_bytes <= kMediumBytes ? 1 : 2;
  r.t_submit = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return fail(TTC_ERR_INVALID_ARG, "server is shutting down");
  if (S->reqs.empty()) S->first_submit = r.t_submit;
  *ticket = int64_t(S->reqs.size());
  if (plan->canon.n == 0) {
    r.state = RQ_DONE;
    r.t_done = r.t_submit;
    S->reqs.push_back(r);
    S->n_completed += 1;
    S->latencies_us.push_back(0.0);
    return TTC_OK;
  }
  S->reqs.push_back(r);
  S->pending.push_back(*ticket);
  S->npending.store(int64_t(S->pending.size()), std::memory_order_release);
  S->cv_sched.notify_one();
  return TTC_OK;
}

ttc_status ttc_server_poll(ttc_server_t S, int64_t ticket, int64_t timeout_us) {
  if (!S) return fail(TTC_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket < 0 || ticket >= int64_t(S->reqs.size())) return fail(TTC_ERR_INVALID_ARG, "no such ticket");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
  while (S->reqs[size_t(ticket)].state != RQ_DONE) {
    if (timeout_us <= 0 || S->cv_poll.wait_until(lk, deadline) == std::cv_status::timeout) {
      if (S->reqs[size_t(ticket)].state == RQ_DONE) break;
      return fail(TTC_ERR_NOT_READY, "request not finished");
    }
  }
  const ttc_status st = S->reqs[size_t(ticket)].status;
  return st == TTC_OK ? TTC_OK : fail(st, "request failed");
}

ttc_status ttc_server_drain(ttc_server_t S, int64_t timeout_us) {
  if (!S) return fail(TTC_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max<int64_t>(0, timeout_us));
  auto idle = [&] { return S->pending.empty() && S->inflight == 0 && S->launching == 0; };
  while (!idle()) {
    if (S->cv_poll.wait_until(lk, deadline) == std::cv_status::timeout && !idle())
      return fail(TTC_ERR_TIMEOUT, "server did not drain in time");
  }
  return TTC_OK;
}

ttc_status ttc_server_stats(ttc_server_t S, ttc_server_stats_t* st) {
  if (!S || !st) return fail(TTC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = int64_t(S->reqs.size());
  st->completed = S->n_completed;
  st->failed = S->n_failed;
  st->epochs = S->n_epochs;
  st->launches = S->n_launches;
  st->bytes = S->done_bytes;
  st->first_submit_s = S->first_submit;
  st->last_complete_s = S->last_complete;
  st->peak_inflight_bytes = S->peak_inflight;
  std::vector<double> l(S->latencies_us);
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l[std::min(l.size() - 1, size_t(q * double(l.size() - 1) + 0.5))]; };
    st->p50_us = pct(0.50);
    st->p90_us = pct(0.90);
    st->p99_us = pct(0.99);
    st->max_us = l.back();
    double sum = 0;
    for (double x : l) sum += x;
    st->mean_us = sum / double(l.size());
  }
  return TTC_OK;
}

ttc_status ttc_server_times(ttc_server_t S, int64_t ticket, double* submit_s, double* admit_s, double* launch_s,
                            double* complete_s) {
  if (!S || !submit_s || !admit_s || !launch_s || !complete_s) return fail(TTC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticket < 0 || ticket >= int64_t(S->reqs.size())) return fail(TTC_ERR_INVALID_ARG, "no such ticket");
  const Req& r = S->reqs[size_t(ticket)];
  *submit_s = r.t_submit;
  *admit_s = r.t_admit;
  *launch_s = r.t_launch;
  *complete_s = r.t_done;
  return r.state == RQ_DONE ? TTC_OK : fail(TTC_ERR_NOT_READY, "request not finished");
}

ttc_status ttc_server_destroy(ttc_server_t S) {
  if (!S) return fail(TTC_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->stop_flag.store(true);
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  if (S->sched.joinable()) S->sched.join();
  if (S->compl_thread.joinable()) S->compl_thread.join();
  cudaSetDevice(S->dev);
  free_lanes(S->lanes);
  for (auto ev : S->free_events) cudaEventDestroy(ev);
  delete S;
  return TTC_OK;
}

}  // extern "C"

// ------------------------------------------------------------- testing hooks

extern "C" ttc_status ttc_debug_server_set_watchdog(ttc_server_t S, double seconds) {
  if (!S || !(seconds > 0)) return fail(TTC_ERR_INVALID_ARG, "bad server or watchdog");
  std::lock_guard<std::mutex> lk(S->mu);
  S->watchdog_s = seconds;
  return TTC_OK;
}

extern "C" ttc_status ttc_debug_server_submit_delay(ttc_server_t S, int64_t microseconds, int64_t* ticket) {
  if (!S || !ticket || microseconds < 0 || microseconds > 10000000)
    return fail(TTC_ERR_INVALID_ARG, "bad server, ticket or delay (0..10 s)");
  Req r;
  r.plan = nullptr;
  r.A = nullptr;
  r.B = nullptr;
  r.bytes = 0;
  r.alg_bytes = 0;
  r.tiles = -1;
  r.cls = S->small_tiles == 0 ? 0 : 2;
  r.delay_ns = uint64_t(microseconds) * 1000u;
  r.t_submit = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return fail(TTC_ERR_INVALID_ARG, "server is shutting down");
  if (S->reqs.empty()) S->first_submit = r.t_submit;
  *ticket = int64_t(S->reqs.size());
  S->reqs.push_back(r);
  S->pending.push_back(*ticket);
  S->npending.store(int64_t(S->pending.size()), std::memory_order_release);
  S->cv_sched.notify_one();
  return TTC_OK;
}
