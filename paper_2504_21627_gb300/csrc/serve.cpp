// Serving loop: continuous batching of query requests over a pool of CUDA
// streams. A request waits in a FIFO queue until a stream can take it and
// its scratch fits the context's memory budget; it is then launched on that
// stream, so requests admitted later overlap on the device with those
// already running. A stream takes up to kDepth requests: one behind another
// in stream order when the stream's scratch already fits it, so that the
// device moves from one to the next without a host call in between. Completion is observed through CUDA events; lsnif_poll
// never blocks past its timeout. Each stream has its own device error word:
// a failed device-side check (an unknown object handle, a bounded wait that
// gave up) is copied to page-locked host memory behind the request's kernels
// and charged to that request alone, without a blocking read.
#include <cuda_runtime.h>

#include <chrono>
#include <thread>

#include "runtime.h"

using namespace lsnif;

namespace lsnif {

constexpr int kStreams = 4;
constexpr int kDepth = 2;  // requests in flight per stream
constexpr size_t kMaxQueued = 4096;

enum ReqState { kQueued, kRunning, kDone };

struct Request {
  uint64_t ticket = 0;
  lsnif_rays rays{};
  lsnif_hits hits{};
  int precision = 0;
  ReqState state = kQueued;
  int stream = -1;
  int rc = LSNIF_OK;
  double submit_us = 0, start_us = 0, done_us = 0;
  cudaEvent_t ev_ready = nullptr;  // the caller's stream reached submit: inputs are ready
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  float gpu_ms = 0.f;
  int err_idx = -1;  // which of its stream's host error words receives its device errors
};

struct StreamSlot {
  cudaStream_t s = nullptr;
  Workspace ws;
  std::deque<Request *> inflight;  // launched, in stream order
  int *d_err = nullptr;            // this stream's device error word (kept at 0 between requests)
  volatile int *h_err = nullptr;   // kDepth page-locked words, one per request in flight (round robin)
  uint64_t launched = 0;
};

struct Server {
  StreamSlot slots[kStreams];
  std::deque<Request *> queue;
  std::map<uint64_t, Request *> all;
  uint64_t next_ticket = 1;
};

static double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void server_shutdown(lsnif_ctx *ctx) {
  Server *sv = ctx->server;
  if (!sv) return;
  for (auto &sl : sv->slots) {
    if (sl.s) {
      cudaStreamSynchronize(sl.s);
      cudaStreamDestroy(sl.s);
    }
    free_workspace(ctx, &sl.ws);
    if (sl.d_err) dev_free(ctx, sl.d_err);
    if (sl.h_err) cudaFreeHost((void *)sl.h_err);
  }
  for (auto &kv : sv->all) {
    if (kv.second->ev_ready) cudaEventDestroy(kv.second->ev_ready);
    if (kv.second->ev_start) cudaEventDestroy(kv.second->ev_start);
    if (kv.second->ev_done) cudaEventDestroy(kv.second->ev_done);
    delete kv.second;
  }
  delete sv;
  ctx->server = nullptr;
}

static int server_get(lsnif_ctx *ctx, Server **out) {
  if (!ctx->server) {
    Server *sv = new Server();
    for (auto &sl : sv->slots) {
      void *d = nullptr, *h = nullptr;
      int rc = LSNIF_OK;
      if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(LSNIF_ERR_CUDA, "serving: cannot create streams");
      } else if ((rc = dev_alloc(ctx, sizeof(int), &d, "serving error word")) == LSNIF_OK) {
        sl.d_err = static_cast<int *>(d);
        if (cudaMemset(sl.d_err, 0, sizeof(int)) != cudaSuccess ||
            cudaHostAlloc(&h, kDepth * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
          cudaGetLastError();
          rc = fail(LSNIF_ERR_CUDA, "serving: cannot set up the error words");
        } else {
          sl.h_err = static_cast<volatile int *>(h);
          for (int k = 0; k < kDepth; ++k) sl.h_err[k] = 0;
        }
      }
      if (rc != LSNIF_OK) {
        ctx->server = sv;
        server_shutdown(ctx);
        return rc;
      }
    }
    ctx->server = sv;
  }
  *out = ctx->server;
  return LSNIF_OK;
}

// Observe finished requests (in stream order), then admit queued ones in
// FIFO order while a stream can take them and memory allows.
static void advance(lsnif_ctx *ctx, Server *sv) {
  for (auto &sl : sv->slots) {
    while (!sl.inflight.empty()) {
      Request *r = sl.inflight.front();
      cudaError_t q = cudaEventQuery(r->ev_done);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->rc = fail(LSNIF_ERR_CUDA, "serving: request %llu failed on the device", (unsigned long long)r->ticket);
      } else {
        cudaEventElapsedTime(&r->gpu_ms, r->ev_start, r->ev_done);
        // the stream's error word, copied behind the request's kernels (ev_done follows the copy)
        const int h = sl.h_err[r->err_idx];
        if (h) {
          sl.h_err[r->err_idx] = 0;
          r->rc = fail(LSNIF_ERR_DEVICE_CHECK, "serving: request %llu: a kernel reported a failed check (0x%x)",
                       (unsigned long long)r->ticket, h);
        }
      }
      r->state = kDone;
      r->done_us = now_us();
      sl.inflight.pop_front();
    }
  }
  while (!sv->queue.empty()) {
    Request *r = sv->queue.front();
    int H = 0, n_in = 0, n_slots = std::max(ctx->n_slots_used, 1);
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) {
        H = std::max(H, ctx->slots[s]->cfg.H);
        n_in = std::max(n_in, ctx->slots[s]->d.n_in);
      }
    const int nin_q = r->precision == LSNIF_FP32_PLAIN ? n_in : 0;
    auto fits = [&](const StreamSlot &sl) {
      return sl.ws.base && r->rays.n <= sl.ws.cap_rays && H <= sl.ws.cap_H && n_slots <= sl.ws.cap_slots &&
             nin_q <= sl.ws.cap_nin;
    };
    // an idle stream first (its scratch may be regrown); else a stream with
    // room in its depth whose scratch already fits (no regrowth while busy)
    int pick = -1;
    for (int i = 0; i < kStreams && pick < 0; ++i)
      if (sv->slots[i].inflight.empty()) pick = i;
    for (int i = 0; i < kStreams && pick < 0; ++i)
      if ((int)sv->slots[i].inflight.size() < kDepth && fits(sv->slots[i])) pick = i;
    if (pick < 0) return;
    StreamSlot &sl = sv->slots[pick];
    int running = 0;
    for (auto &s2 : sv->slots) running += (int)s2.inflight.size();
    // memory admission: the request's scratch must fit the budget; idle
    // streams give their scratch back before a request is refused
    int rc = LSNIF_OK;
    if (!fits(sl)) {
      cudaStreamSynchronize(sl.s);
      free_workspace(ctx, &sl.ws);
      size_t need = workspace_bytes(r->rays.n, H, n_slots, nin_q);
      if (ctx->budget && ctx->used + need > ctx->budget) {
        for (auto &s2 : sv->slots)
          if (s2.inflight.empty() && s2.ws.base) free_workspace(ctx, &s2.ws);
      }
      if (ctx->budget && ctx->used + need > ctx->budget) {
        if (running) return;  // wait for memory to free up
        rc = fail(LSNIF_ERR_OVER_BUDGET, "serving: request of %lld rays needs %zu bytes of scratch",
                  (long long)r->rays.n, need);
      } else {
        rc = ensure_workspace(ctx, &sl.ws, r->rays.n, H, n_slots, nin_q);
        if (rc == LSNIF_ERR_OVER_BUDGET && running) return;
      }
    }
    sv->queue.pop_front();
    r->start_us = now_us();
    if (rc == LSNIF_OK) {
      r->err_idx = (int)(sl.launched++ % kDepth);
      cudaStreamWaitEvent(sl.s, r->ev_ready, 0);   // after the caller's writes to the buffers
      cudaEventRecord(r->ev_start, sl.s);
      rc = run_query(ctx, &sl.ws, &r->rays, &r->hits, r->precision, sl.s, false, sl.d_err);
      if (rc == LSNIF_OK) {
        // hand the error word to the host and clear it for the stream's next request
        cudaError_t e = cudaMemcpyAsync((void *)(sl.h_err + r->err_idx), sl.d_err, sizeof(int),
                                        cudaMemcpyDeviceToHost, sl.s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_err, 0, sizeof(int), sl.s);
        if (e != cudaSuccess) rc = cuda_fail(e, "serving: error word");
      }
      cudaEventRecord(r->ev_done, sl.s);
    }
    if (rc != LSNIF_OK) {
      r->rc = rc;
      r->state = kDone;
      r->done_us = now_us();
      continue;
    }
    r->state = kRunning;
    r->stream = pick;
    sl.inflight.push_back(r);
  }
}

}  // namespace lsnif

extern "C" int lsnif_submit(lsnif_ctx *ctx, const lsnif_rays *rays, lsnif_hits *hits, int precision,
                            void *stream, uint64_t *ticket) {
  if (!ctx || !rays || !hits || !ticket) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_submit: NULL argument");
  if (!valid_precision(precision)) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_submit: unknown precision %d", precision);
  if (rays->n < 0) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_submit: n < 0");
  cudaSetDevice(ctx->device);
  Server *sv;
  int rc = server_get(ctx, &sv);
  if (rc) return rc;
  if (sv->queue.size() >= kMaxQueued) return fail(LSNIF_ERR_BUSY, "lsnif_submit: %zu requests queued", sv->queue.size());
  if (ctx->budget) {
    int H = 0, n_in = 0;
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) {
        H = std::max(H, ctx->slots[s]->cfg.H);
        n_in = std::max(n_in, ctx->slots[s]->d.n_in);
      }
    size_t objects = 0;
    for (int s = 0; s < ctx->n_slots_used; ++s)
      if (ctx->slots[s]) objects += ctx->slots[s]->device_bytes;
    size_t need = workspace_bytes(rays->n, H, std::max(ctx->n_slots_used, 1),
                                  precision == LSNIF_FP32_PLAIN ? n_in : 0);
    if (objects + need > ctx->budget)
      return fail(LSNIF_ERR_OVER_BUDGET, "lsnif_submit: a request of %lld rays can never fit the budget",
                  (long long)rays->n);
  }
  Request *r = new Request();
  r->ticket = sv->next_ticket++;
  r->rays = *rays;
  r->hits = *hits;
  r->precision = precision;
  r->submit_us = now_us();
  cudaEventCreateWithFlags(&r->ev_ready, cudaEventDisableTiming);
  cudaEventRecord(r->ev_ready, (cudaStream_t)stream);
  cudaEventCreate(&r->ev_start);
  cudaEventCreate(&r->ev_done);
  sv->queue.push_back(r);
  sv->all[r->ticket] = r;
  *ticket = r->ticket;
  advance(ctx, sv);
  return LSNIF_OK;
}

extern "C" int lsnif_poll(lsnif_ctx *ctx, uint64_t ticket, int64_t timeout_us, lsnif_req_stats *st) {
  if (!ctx) return fail(LSNIF_ERR_INVALID_ARG, "lsnif_poll: ctx is NULL");
  Server *sv = ctx->server;
  if (!sv) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_poll: unknown ticket %llu", (unsigned long long)ticket);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(LSNIF_ERR_BAD_HANDLE, "lsnif_poll: unknown ticket %llu", (unsigned long long)ticket);
  cudaSetDevice(ctx->device);
  Request *r = it->second;
  const double t_end = now_us() + (double)std::max<int64_t>(timeout_us, 0);
  for (;;) {
    advance(ctx, sv);
    if (r->state == kDone) break;
    if (now_us() >= t_end) return timeout_us <= 0 ? LSNIF_PENDING : fail(LSNIF_ERR_TIMEOUT, "lsnif_poll: timeout");
    std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
  int rc = r->rc;
  if (st) {
    st->submit_us = r->submit_us;
    st->start_us = r->start_us;
    st->done_us = r->done_us;
    st->gpu_ms = r->gpu_ms;
    st->n_rays = r->rays.n;
  }
  cudaEventDestroy(r->ev_ready);
  cudaEventDestroy(r->ev_start);
  cudaEventDestroy(r->ev_done);
  sv->all.erase(it);
  delete r;
  return rc;
}

extern "C" int64_t lsnif_pending(lsnif_ctx *ctx) {
  if (!ctx || !ctx->server) return 0;
  return (int64_t)ctx->server->all.size();
}
