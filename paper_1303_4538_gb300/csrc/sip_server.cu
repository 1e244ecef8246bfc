// sip_server.cu -- continuous-batching request loop over the SIP solver.
//
// A server owns `max_slots` worker slots, each with its own CUDA stream and
// solver context.  Requests (one block each: pressure-correction or momentum
// systems of any size, Sec. 4.1) queue in arrival order; a free slot admits
// the oldest queued request whose estimated device footprint fits in what is
// left of the HBM budget, builds its plan (coefficient copies and factors stay
// on the device for the whole solve), solves to the request's tolerance and
// releases the plan.  Slots run concurrently, so requests that arrive while
// others are on the GPU start as soon as a slot and memory free up and their
// kernels overlap on the device.  The sweep kernels of one launch only wait
// on CTAs of the same launch that claimed earlier tiles and are already
// running, so concurrent launches from different slots cannot block one
// another.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sip.h"
#include "sip_internal.h"

namespace {

struct Request {
  uint64_t ticket;
  sip_block_desc desc;
  sip_options opt;
  double rtol;
  int max_iters;
  size_t footprint;
};

struct Result {
  int done = 0;
  int status = SIP_OK;
  int iters = 0;
  double relres = -1.0;
};

// Device bytes a plan of this block needs (records, vectors, the temporary
// factorisation input, faces and control), with a margin.
size_t estimate_footprint(const sip_block_desc &d, const sip_options &o) {
  const double n = (double)d.nx * d.ny * d.nz;
  const bool sym = d.symmetric != 0;
  double per;
  if (o.mode == SIP_MODE_F64) per = (sym ? 64 : 96) + 32 + 24 + 64;
  else if (o.mode == SIP_MODE_F32) per = (sym ? 32 : 48) + 16 + 16 + 12 + 64;
  else per = (sym ? 32 : 48) + 16 + 16 + 12 + 64 + (d.coef_dtype ? 0 : (sym ? 32 : 64));
  const double faces = 2.0 * n * 48.0 / 8.0;  // face words: small next to the cells
  return (size_t)(n * per + faces) + (size_t)(16u << 20);
}

}  // namespace

struct sip_server {
  int device = 0;
  size_t budget = 0, in_use = 0, peak_in_use = 0;
  uint64_t submitted = 0, completed = 0, failed = 0;
  double busy_ms = 0;
  std::vector<std::chrono::steady_clock::time_point> started;  // per slot: admission of its request
  std::vector<char> running;                                    // per slot: a request is on it
  int max_slots = 0;
  size_t queue_cap = 4096;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, Result> results;
  std::vector<std::thread> workers;
};

namespace {

void slot_loop(sip_server *s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  sip_ctx *ctx = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                  sip_create(&ctx, s->device, stream) == SIP_OK;
  // the slot's pool keeps its fixed cache only: requests are budgeted
  if (ok) sipk::ctx_keep_peak(ctx, false);
  for (;;) {
    Request r{};
    r.ticket = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // the oldest request that fits in the free budget (a request larger than
      // the whole budget is admitted alone, when nothing else is in flight)
      auto pick = [&]() -> bool {
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          const bool fits = s->in_use + it->footprint <= s->budget || (s->in_use == 0 && it == s->queue.begin());
          if (fits) {
            r = *it;
            s->queue.erase(it);
            s->in_use += r.footprint;
            s->peak_in_use = std::max(s->peak_in_use, s->in_use);
            s->running[slot] = 1;
            s->started[slot] = std::chrono::steady_clock::now();
            return true;
          }
          break;  // arrival order: later requests wait behind the oldest
        }
        return false;
      };
      // on stop, queued requests still run (drain) before the slot exits
      s->cv.wait(lk, [&] { return pick() || (s->stopping && s->queue.empty()); });
      if (r.ticket == 0) break;
    }
    Result res;
    res.done = 1;
    if (!ok) {
      res.status = SIP_ERR_CUDA;
    } else {
      sip_plan *plan = nullptr;
      int rc = sip_factor(ctx, &r.desc, 1, nullptr, 0, &r.opt, &plan);
      if (rc == SIP_OK) {
        rc = sip_solve(plan, r.rtol, r.max_iters, &res.iters, &res.relres);
        sip_plan_destroy(plan);
      }
      res.status = rc;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r.footprint;
      s->results[r.ticket] = res;
      s->running[slot] = 0;
      s->completed += 1;
      s->failed += res.status != SIP_OK;
      s->busy_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->started[slot]).count();
    }
    s->cv.notify_all();
  }
  if (ctx) sip_destroy(ctx);
  if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int sip_server_start(sip_ctx *ctx, size_t hbm_budget_bytes, int max_slots, sip_server **out) {
  if (!ctx || !out || max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0) return SIP_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SIP_ERR_NO_DEVICE;
  sip_server *s = new sip_server();
  s->device = dev;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->started.assign(max_slots, std::chrono::steady_clock::time_point());
  s->running.assign(max_slots, 0);
  for (int q = 0; q < max_slots; ++q) s->workers.emplace_back(slot_loop, s, q);
  *out = s;
  return SIP_OK;
}

int sip_server_submit(sip_server *s, const sip_block_desc *blk, const sip_options *opt, double rtol, int max_iters,
                      uint64_t *ticket) {
  if (!s || !blk || !ticket || max_iters < 0 || !(rtol >= 0.0)) return SIP_ERR_INVALID_ARG;
  Request r;
  r.desc = *blk;
  if (opt) r.opt = *opt;
  else sip_default_options(&r.opt);
  r.rtol = rtol;
  r.max_iters = max_iters;
  r.footprint = estimate_footprint(r.desc, r.opt);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return SIP_ERR_INVALID_ARG;
    if (s->queue.size() >= s->queue_cap) return SIP_ERR_BUSY;
    r.ticket = s->next_ticket++;
    s->queue.push_back(r);
    s->submitted += 1;
    s->results[r.ticket] = Result();
    *ticket = r.ticket;
  }
  s->cv.notify_all();
  return SIP_OK;
}

int sip_server_poll(sip_server *s, uint64_t ticket, int *done, int *status, int *iters, double *relres) {
  if (!s) return SIP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return SIP_ERR_NOT_FOUND;
  const Result &r = it->second;
  if (done) *done = r.done;
  if (status) *status = r.status;
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  if (r.done) s->results.erase(it);  // a finished ticket is reported once
  return SIP_OK;
}

int sip_server_get_stats(sip_server *s, sip_server_stats *out) {
  if (!s || !out) return SIP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (uint32_t)s->queue.size();
  out->slots = (uint32_t)s->max_slots;
  out->budget_bytes = s->budget;
  out->in_use_bytes = s->in_use;
  out->peak_in_use_bytes = s->peak_in_use;
  out->busy_ms = s->busy_ms;
  const auto now = std::chrono::steady_clock::now();
  for (int q = 0; q < s->max_slots; ++q)
    if (s->running[q]) {
      out->running += 1;
      out->oldest_running_ms =
          std::max(out->oldest_running_ms, std::chrono::duration<double, std::milli>(now - s->started[q]).count());
    }
  return SIP_OK;
}

int sip_server_stop(sip_server *s) {
  if (!s) return SIP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
  return SIP_OK;
}

}  // extern "C"
