// serve.cu -- the serving runtime: continuous batching of sort requests.
//
// rsort_submit queues a request (caller-owned device buffers) and returns a
// ticket.  A runtime thread per context keeps up to `serve_slots` batches in
// flight, one per CUDA stream, each with its own scratch workspace:
//   - requests of at most `serve_alone_min` keys are grouped (same key type,
//     FIFO order, up to `serve_batch_keys` keys) into one batch: a gather
//     kernel copies their keys into one buffer, one segmented robust sort
//     (rsort_segmented's launch sequence) sorts every request as a segment,
//     and a scatter kernel writes keys and segment-local permutations back to
//     each request's buffers;
//   - larger requests run the plain sort (rsort_sort's launch sequence) as a
//     batch of their own.
// A batch is admitted when a slot is free and its scratch fits the context's
// HBM budget next to the batches in flight; requests that arrive while others
// run are admitted as slots and memory free up, so their work overlaps on the
// device.  Completion is observed by a host function enqueued after the batch
// (behind an asynchronous read-back of the batch's device error word), which
// stamps each request's latency.  Results never depend on the batch a request
// lands in: every request is sorted as its own segment, and the output of the
// robust sort is unique.
// The runtime keeps the record (status, latency) of the last `serve_history`
// finished requests and forgets older ones, so a server that runs for
// millions of requests holds bounded host memory.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace rsort {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = 8;
constexpr uint32_t kMaxBatchRequests = 65536;

struct ReqDesc {  // device-side descriptor of one batched request
  const uint64_t* in;
  uint64_t* out;
  uint32_t* perm;
  uint64_t off;  // first position in the batch buffers
  uint64_t n;
};

enum class RState { Queued, Running, Done, Cancelled, Failed };

struct Req {
  rsort_request r{};
  RState state = RState::Queued;
  rsort_status status = RSORT_PENDING;
  Clock::time_point t_submit, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  Workspace ws;                   // sort scratch
  Workspace bws;                  // batch buffers
  ReqDesc* h_desc = nullptr;      // pinned, kMaxBatchRequests entries
  uint64_t* h_off = nullptr;      // pinned, kMaxBatchRequests + 1 entries
  uint32_t* h_err = nullptr;      // pinned device-error word of the last batch
  bool busy = false;
  std::vector<uint64_t> tickets;  // requests of the batch in flight
  uint64_t keys = 0;
};

__global__ void k_gather(const ReqDesc* desc, uint32_t nreq, const uint64_t* offsets, uint64_t n,
                         uint64_t* keys) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nreq;  // last request with offset <= j
    while (lo + 1 < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= j) lo = mid; else hi = mid;
    }
    const ReqDesc& d = desc[lo];
    keys[j] = d.in[j - d.off];
  }
}

__global__ void k_scatter_back(const ReqDesc* desc, uint32_t nreq, const uint64_t* offsets,
                               uint64_t n, const uint64_t* keys, const uint32_t* perm) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nreq;
    while (lo + 1 < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (offsets[mid] <= j) lo = mid; else hi = mid;
    }
    const ReqDesc& d = desc[lo];
    d.out[j - d.off] = keys[j];
    d.perm[j - d.off] = perm[j];
  }
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct BatchLayout {
  size_t off_keys_in, off_keys_out, off_perm, off_offsets, off_desc, total;
};

BatchLayout batch_layout(uint64_t n, uint32_t nreq) {
  BatchLayout b;
  size_t o = 0;
  b.off_keys_in = o; o = align_up(o + n * 8, 256);
  b.off_keys_out = o; o = align_up(o + n * 8, 256);
  b.off_perm = o; o = align_up(o + n * 4, 256);
  b.off_offsets = o; o = align_up(o + (size_t)(nreq + 1) * 8, 256);
  b.off_desc = o; o = align_up(o + (size_t)nreq * sizeof(ReqDesc), 256);
  b.total = o;
  return b;
}

}  // namespace

struct Server {
  rsort_ctx* c = nullptr;
  int nslots = 4;
  uint64_t batch_keys = 1ull << 24;
  uint64_t alone_min = 1ull << 20;
  std::mutex mu;
  std::condition_variable cv;       // wakes the runtime thread
  std::condition_variable done_cv;  // wakes waiters
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t history = 1ull << 20;  // finished requests whose record is kept
  std::deque<uint64_t> finished;  // their tickets, oldest first
  Slot slots[kMaxSlots];
  std::thread th;
  bool stop = false;
  uint64_t next_ticket = 1;
  // statistics
  std::vector<double> lat_ns;  // latencies of the last `history` completions (a ring)
  size_t lat_next = 0;         // ring slot the next latency overwrites once full
  uint64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, batches = 0;
  uint64_t batched_requests = 0, keys_done = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;

  struct CbArg {
    Server* s;
    int slot;
  } cb[kMaxSlots];

  static void CUDART_CB on_done(void* p) {
    CbArg* a = static_cast<CbArg*>(p);
    a->s->finish_slot(a->slot);
  }

  // A request reached a final state and left the queue (lock held): it joins
  // the finished records, and the oldest record beyond `history` is dropped.
  void retire(uint64_t t) {
    finished.push_back(t);
    while (finished.size() > history) {
      reqs.erase(finished.front());
      finished.pop_front();
    }
  }

  void record_latency(double ns) {
    if (lat_ns.size() < history) {
      lat_ns.push_back(ns);
    } else {
      lat_ns[lat_next] = ns;
      lat_next = (lat_next + 1) % history;
    }
  }

  // Called from the CUDA callback thread: no CUDA calls here.
  void finish_slot(int si) {
    std::lock_guard<std::mutex> lk(mu);
    Slot& sl = slots[si];
    const Clock::time_point now = Clock::now();
    const bool err = *sl.h_err != 0;
    for (uint64_t t : sl.tickets) {
      Req& q = reqs[t];
      q.t_done = now;
      if (err) {
        q.state = RState::Failed;
        q.status = RSORT_EDEVICE;
        ++failed;
      } else {
        q.state = RState::Done;
        q.status = RSORT_OK;
        ++completed;
        keys_done += q.r.n;
        record_latency(
            (double)std::chrono::duration_cast<std::chrono::nanoseconds>(now - q.t_submit).count());
      }
      retire(t);
    }
    t_last = now;
    sl.tickets.clear();
    sl.busy = false;
    cv.notify_all();
    done_cv.notify_all();
  }

  int free_slot() const {
    for (int i = 0; i < nslots; ++i)
      if (!slots[i].busy) return i;
    return -1;
  }
  int busy_slots() const {
    int b = 0;
    for (int i = 0; i < nslots; ++i) b += slots[i].busy ? 1 : 0;
    return b;
  }

  // Scratch a batch of `keys` keys in `nreq` requests needs (alone: plain sort).
  size_t footprint(bool alone, uint64_t keys, uint32_t nreq, uint32_t p) {
    if (alone) return sort_scratch_bytes(c, keys, p);
    return segmented_scratch_bytes(c, keys, nreq) + batch_layout(keys, nreq).total;
  }

  // Whether ticket t is waiting in the queue (lock held); a cancelled entry
  // that leaves the queue here is retired.
  bool still_queued(uint64_t t) {
    const auto it = reqs.find(t);
    if (it == reqs.end()) return false;
    if (it->second.state == RState::Queued) return true;
    retire(t);
    return false;
  }

  // Forms the next batch from the queue front (lock held).  Returns false if
  // the queue holds only cancelled entries.
  bool form_batch(std::vector<uint64_t>& out, bool& alone, uint64_t& keys) {
    out.clear();
    keys = 0;
    while (!queue.empty() && !still_queued(queue.front())) queue.pop_front();
    if (queue.empty()) return false;
    const uint64_t first = queue.front();
    const Req& f = reqs[first];
    alone = f.r.n > alone_min;
    if (alone) {
      out.push_back(first);
      keys = f.r.n;
      queue.pop_front();
      return true;
    }
    std::deque<uint64_t> rest;
    for (uint64_t t : queue) {
      if (!still_queued(t)) continue;
      const Req& q = reqs[t];
      const bool fits = q.r.type == f.r.type && q.r.n <= alone_min &&
                        keys + q.r.n <= batch_keys && out.size() < kMaxBatchRequests;
      if (fits || out.empty()) {
        out.push_back(t);
        keys += q.r.n;
      } else {
        rest.push_back(t);
      }
    }
    queue.swap(rest);
    return true;
  }

  // Enqueues one batch on its slot's stream (called without the lock: rq is
  // a private copy of the requests' descriptors).
  rsort_status launch(int si, const std::vector<rsort_request>& rq, bool alone, uint64_t keys) {
    Slot& sl = slots[si];
    LaunchEnv e = env_of(c, sl.stream);
    e.timer = nullptr;  // the profiling timer belongs to the synchronous entry points
    DevState* st = nullptr;
    rsort_status rs;
    if (alone) {
      const rsort_request& r = rq[0];
      rs = enqueue_sort(c, sl.ws, e, r.type, r.d_keys_in, r.d_keys_out, r.d_perm_out, r.n,
                        r.p_virtual ? r.p_virtual : 1, r.seed, &st);
    } else {
      const uint32_t nreq = (uint32_t)rq.size();
      const BatchLayout bl = batch_layout(keys, nreq);
      rs = ensure_workspace(c, sl.bws, bl.total, sl.stream);
      if (rs != RSORT_OK) return rs;
      unsigned char* base = static_cast<unsigned char*>(sl.bws.arena);
      uint64_t* d_in = (uint64_t*)(base + bl.off_keys_in);
      uint64_t* d_out = (uint64_t*)(base + bl.off_keys_out);
      uint32_t* d_perm = (uint32_t*)(base + bl.off_perm);
      uint64_t* d_off = (uint64_t*)(base + bl.off_offsets);
      ReqDesc* d_desc = (ReqDesc*)(base + bl.off_desc);
      uint64_t o = 0;
      for (uint32_t i = 0; i < nreq; ++i) {
        const rsort_request& r = rq[i];
        sl.h_desc[i] = ReqDesc{(const uint64_t*)r.d_keys_in, (uint64_t*)r.d_keys_out,
                               r.d_perm_out, o, r.n};
        sl.h_off[i] = o;
        o += r.n;
      }
      sl.h_off[nreq] = o;
      cudaMemcpyAsync(d_desc, sl.h_desc, (size_t)nreq * sizeof(ReqDesc), cudaMemcpyHostToDevice,
                      sl.stream);
      cudaMemcpyAsync(d_off, sl.h_off, (size_t)(nreq + 1) * 8, cudaMemcpyHostToDevice,
                      sl.stream);
      const int grid = (int)std::min<uint64_t>((keys + 255) / 256 + 1, (uint64_t)c->num_sms * 8);
      k_gather<<<grid, 256, 0, sl.stream>>>(d_desc, nreq, d_off, keys, d_in);
      ++c->launches;
      const rsort_request& r0 = rq[0];
      rs = enqueue_segmented(c, sl.ws, e, r0.type, d_in, d_out, d_perm, keys, d_off, nreq,
                             r0.seed, &st);
      if (rs != RSORT_OK) return rs;
      k_scatter_back<<<grid, 256, 0, sl.stream>>>(d_desc, nreq, d_off, keys, d_out, d_perm);
      ++c->launches;
    }
    if (rs != RSORT_OK) return rs;
    cudaMemcpyAsync(sl.h_err, &st->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, sl.stream);
    if (cudaLaunchHostFunc(sl.stream, &Server::on_done, &cb[si]) != cudaSuccess) {
      cudaGetLastError();
      return RSORT_ECUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return RSORT_ECUDA;
    return RSORT_OK;
  }

  void fail(const std::vector<uint64_t>& batch, rsort_status s) {
    const Clock::time_point now = Clock::now();
    for (uint64_t t : batch) {
      Req& q = reqs[t];
      q.state = RState::Failed;
      q.status = s;
      q.t_done = now;
      ++failed;
      retire(t);
    }
    done_cv.notify_all();
  }

  void run() {
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    std::vector<uint64_t> batch;
    while (true) {
      cv.wait(lk, [&] { return stop || (!queue.empty() && free_slot() >= 0); });
      if (stop) break;
      const int si = free_slot();
      bool alone = false;
      uint64_t keys = 0;
      if (!form_batch(batch, alone, keys)) continue;
      // admission by HBM budget: the batch's scratch next to the batches in flight
      const Req& f = reqs[batch[0]];
      const size_t need = footprint(alone, keys, (uint32_t)batch.size(), f.r.p_virtual);
      if (c->budget) {
        uint64_t held_busy = c->ws.bytes;
        for (int i = 0; i < nslots; ++i)
          if (slots[i].busy) held_busy += slots[i].ws.bytes + slots[i].bws.bytes;
        if (held_busy + need > c->budget) {
          const int b0 = busy_slots();
          if (b0 > 0) {
            // wait for memory: put the batch back at the queue front in order,
            // and wait until a batch in flight completes
            for (auto it = batch.rbegin(); it != batch.rend(); ++it) queue.push_front(*it);
            cv.wait(lk, [&] { return stop || busy_slots() < b0; });
            continue;
          }
        }
        // release the scratch of idle slots so this batch can grow into it
        for (int i = 0; i < nslots; ++i) {
          if (!slots[i].busy && i != si) {
            release_workspace(c, slots[i].ws, slots[i].stream);
            release_workspace(c, slots[i].bws, slots[i].stream);
          }
        }
      }
      std::vector<rsort_request> rq;
      rq.reserve(batch.size());
      for (uint64_t t : batch) {
        reqs[t].state = RState::Running;
        rq.push_back(reqs[t].r);
      }
      Slot& sl = slots[si];
      sl.busy = true;
      sl.tickets = batch;
      sl.keys = keys;
      ++batches;
      batched_requests += batch.size();
      lk.unlock();
      const rsort_status rs = launch(si, rq, alone, keys);
      lk.lock();
      if (rs != RSORT_OK) {
        // nothing of this batch will complete: fail its requests (the slot's
        // host function was not enqueued)
        sl.busy = false;
        sl.tickets.clear();
        fail(batch, rs);
      }
    }
  }
};

}  // namespace rsort

using namespace rsort;

namespace {

rsort::Server* get_server(rsort_ctx* c, rsort_status* err) {
  std::lock_guard<std::mutex> lk(c->server_mu);
  if (c->server) return c->server;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  Server* s = new Server();
  s->c = c;
  s->nslots = std::max(1, std::min(kMaxSlots, c->serve_slots));
  s->batch_keys = c->serve_batch_keys;
  s->alone_min = c->serve_alone_min;
  s->history = std::max<uint64_t>(1, c->serve_history);
  bool ok = true;
  for (int i = 0; i < s->nslots && ok; ++i) {
    Slot& sl = s->slots[i];
    ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaMallocHost(&sl.h_desc, sizeof(ReqDesc) * kMaxBatchRequests) == cudaSuccess &&
         cudaMallocHost(&sl.h_off, sizeof(uint64_t) * (kMaxBatchRequests + 1)) == cudaSuccess &&
         cudaMallocHost(&sl.h_err, sizeof(uint32_t)) == cudaSuccess;
    s->cb[i] = Server::CbArg{s, i};
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    *err = RSORT_ECUDA;
    for (int i = 0; i < s->nslots; ++i) {
      if (s->slots[i].stream) cudaStreamDestroy(s->slots[i].stream);
      if (s->slots[i].h_desc) cudaFreeHost(s->slots[i].h_desc);
      if (s->slots[i].h_off) cudaFreeHost(s->slots[i].h_off);
      if (s->slots[i].h_err) cudaFreeHost(s->slots[i].h_err);
    }
    delete s;
    return nullptr;
  }
  s->th = std::thread([s] { s->run(); });
  c->server = s;
  return s;
}

bool terminal(RState st) {
  return st == RState::Done || st == RState::Failed || st == RState::Cancelled;
}

rsort_status report(const Req& q, uint64_t* latency_ns_out) {
  switch (q.state) {
    case RState::Done:
      if (latency_ns_out)
        *latency_ns_out = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                              q.t_done - q.t_submit).count();
      return RSORT_OK;
    case RState::Cancelled: return RSORT_ECANCELLED;
    case RState::Failed: return q.status;
    default: return RSORT_PENDING;
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

namespace rsort {

void destroy_server(rsort_ctx* c) {
  Server* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(c->server_mu);
    s = c->server;
    c->server = nullptr;
  }
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  for (int i = 0; i < s->nslots; ++i) {
    Slot& sl = s->slots[i];
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    release_workspace(c, sl.ws, nullptr);
    release_workspace(c, sl.bws, nullptr);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.h_off) cudaFreeHost(sl.h_off);
    if (sl.h_err) cudaFreeHost(sl.h_err);
  }
  cudaGetLastError();
  delete s;
}

}  // namespace rsort

extern "C" {

rsort_status rsort_submit(rsort_ctx* c, const rsort_request* r, uint64_t* ticket_out) {
  if (!c || !r || !ticket_out) return RSORT_EINVAL;
  if (r->type != RSORT_KEY_U64 && r->type != RSORT_KEY_F64) return RSORT_EINVAL;
  if (r->n > 0xFFFFFFFFull || r->p_virtual > (uint32_t)kMaxK) return RSORT_EINVAL;
  if (r->n > 0 && (!r->d_keys_in || !r->d_keys_out || !r->d_perm_out)) return RSORT_EINVAL;
  if (r->n > 0 && r->d_keys_in == r->d_keys_out) return RSORT_EINVAL;
  rsort_status err = RSORT_OK;
  Server* s = get_server(c, &err);
  if (!s) return err;
  // a request that cannot fit the budget even alone is refused now
  const bool alone = r->n > s->alone_min;
  const size_t need = s->footprint(alone, r->n, 1, r->p_virtual);
  if (c->budget && need > c->budget) return RSORT_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  const uint64_t t = s->next_ticket++;
  Req q;
  q.r = *r;
  q.t_submit = Clock::now();
  if (!s->have_first) {
    s->have_first = true;
    s->t_first = q.t_submit;
  }
  ++s->submitted;
  if (r->n == 0) {
    q.state = RState::Done;
    q.status = RSORT_OK;
    q.t_done = q.t_submit;
    ++s->completed;
    s->reqs[t] = q;
    s->retire(t);
  } else {
    s->reqs[t] = q;
    s->queue.push_back(t);
    s->cv.notify_all();
  }
  *ticket_out = t;
  return RSORT_OK;
}

rsort_status rsort_poll(rsort_ctx* c, uint64_t ticket, uint64_t* latency_ns_out) {
  if (!c) return RSORT_EINVAL;
  Server* s = c->server;
  if (!s) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RSORT_EINVAL;
  return report(it->second, latency_ns_out);
}

rsort_status rsort_wait(rsort_ctx* c, uint64_t ticket, uint64_t timeout_ns) {
  if (!c) return RSORT_EINVAL;
  Server* s = c->server;
  if (!s) return RSORT_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RSORT_EINVAL;
  const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
  // the record may be dropped while this thread sleeps (more than
  // serve_history later requests finished): the ticket is then unknown
  const bool done = s->done_cv.wait_until(lk, deadline, [&] {
    const auto i = s->reqs.find(ticket);
    return i == s->reqs.end() || terminal(i->second.state);
  });
  if (!done) return RSORT_ETIMEOUT;
  const auto i = s->reqs.find(ticket);
  if (i == s->reqs.end()) return RSORT_EINVAL;
  return report(i->second, nullptr);
}

rsort_status rsort_cancel(rsort_ctx* c, uint64_t ticket) {
  if (!c) return RSORT_EINVAL;
  Server* s = c->server;
  if (!s) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RSORT_EINVAL;
  Req& q = it->second;
  if (q.state != RState::Queued) return RSORT_EINVAL;  // running or finished
  q.state = RState::Cancelled;
  q.status = RSORT_ECANCELLED;
  q.t_done = Clock::now();
  ++s->cancelled;
  s->done_cv.notify_all();
  return RSORT_OK;
}

rsort_status rsort_get_serve_stats(rsort_ctx* c, rsort_serve_stats* out) {
  if (!c || !out) return RSORT_EINVAL;
  memset(out, 0, sizeof(*out));
  Server* s = c->server;
  if (!s) return RSORT_OK;
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->cancelled = s->cancelled;
    out->failed = s->failed;
    for (uint64_t t : s->queue) {
      const auto i = s->reqs.find(t);
      if (i != s->reqs.end() && i->second.state == RState::Queued) ++out->queued;
    }
    out->inflight_batches = (uint32_t)s->busy_slots();
    out->batches = s->batches;
    out->keys_completed = s->keys_done;
    out->mean_batch_requests = s->batches ? (double)s->batched_requests / s->batches : 0.0;
    if (s->have_first && s->completed)
      out->elapsed_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    lat = s->lat_ns;
  }
  out->p50_us = percentile(lat, 0.50) / 1e3;
  out->p99_us = percentile(lat, 0.99) / 1e3;
  out->max_us = lat.empty() ? 0.0 : *std::max_element(lat.begin(), lat.end()) / 1e3;
  return RSORT_OK;
}

rsort_status rsort_reset_serve_stats(rsort_ctx* c) {
  if (!c) return RSORT_EINVAL;
  Server* s = c->server;
  if (!s) return RSORT_OK;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ns.clear();
  s->lat_next = 0;
  s->submitted = s->completed = s->cancelled = s->failed = s->batches = 0;
  s->batched_requests = s->keys_done = 0;
  s->have_first = false;
  return RSORT_OK;
}

}  // extern "C"
