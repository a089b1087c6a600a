// Continuous-batching request loop.
//
// A worker thread owns the GPU work of all requests:
//   * admission: pending requests are admitted first-come first-served while the device-memory
//     budget allows (a later request may pass an earlier one that does not fit yet).  Requests
//     with at most `small_nnz` nonzeros become slots of the batched solver (their memory is
//     carved from its arena, which counts against the budget); larger ones get their own
//     single-LP handle on their own stream, created and solved asynchronously.
//   * progress: each loop turn advances every batched slot by `iters_per_step` iterations in one
//     launch, while the single-LP handles run concurrently on their streams; finished requests
//     release their memory at once, so waiting requests are admitted in the next turn.
// Results are copied to host buffers owned by the request and handed out by poll.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rhpdhg.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  // owned copy of the problem
  int32_t m_eq = 0, m_ineq = 0, n = 0;
  double obj_offset = 0.0;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col_idx;
  std::vector<double> val, c, rhs, l, u;
  rhpdhg_params params{};
  // placement
  int where = 0;            // 0 pending, 1 batched slot, 2 own handle, 3 done
  int32_t slot = -1;
  rhpdhg_handle *h = nullptr;
  int64_t bytes = 0;
  bool cancel = false;
  // result
  rhpdhg_result res{};
  std::vector<double> x, y, cx, cy;
  Clock::time_point t_submit, t_admit, t_done;

  rhpdhg_problem problem() const {
    rhpdhg_problem p{};
    p.m_eq = m_eq;
    p.m_ineq = m_ineq;
    p.n = n;
    p.memory = RHPDHG_MEM_HOST;
    p.nnz = row_ptr.empty() ? 0 : row_ptr.back();
    p.row_ptr = row_ptr.data();
    p.col_idx = col_idx.data();
    p.val = val.data();
    p.c = c.data();
    p.rhs = rhs.data();
    p.l = l.data();
    p.u = u.data();
    p.obj_offset = obj_offset;
    return p;
  }
};

}  // namespace

struct rhpdhg_server {
  int dev = 0;
  int64_t budget = 0, in_use = 0, small_nnz = 0;
  int32_t iters_per_step = 64;
  rhpdhg_batch *batch = nullptr;
  int64_t arena_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> pending;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::string err;
  // statistics
  int64_t admitted_batched = 0, admitted_single = 0, completed = 0, peak_in_use = 0;
  int64_t steps = 0;
};

namespace {

int64_t single_lp_bytes(const Request &r) {
  // device footprint of a single-LP handle: two copies of the matrix (row and column layouts,
  // FP64 values + int32 indices, plus an FP32 copy in mixed precision, plus padding), the
  // vectors of the iteration, and the create-time transients (the input copy and the CSC)
  const int64_t m = (int64_t)r.m_eq + r.m_ineq, n = r.n;
  const int64_t nnz = r.row_ptr.empty() ? 0 : r.row_ptr.back();
  const int64_t per_nnz = 2 * (8 + 4 + (r.params.precision == 1 ? 4 : 0)) + 2 * 12;
  return nnz * per_nnz + (m + n) * 8 * 24 + (64 << 20);
}

void finish_request(rhpdhg_server *s, Request &r, const rhpdhg_result &res) {
  r.res = res;
  r.where = 3;
  r.t_done = Clock::now();
  s->completed++;
}

void worker_loop(rhpdhg_server *s) {
  cudaSetDevice(s->dev);
  while (!s->stop.load()) {
    bool batched_active = false;
    std::vector<Request *> singles;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // ---- admission (first fit in arrival order) ----
      for (auto it = s->pending.begin(); it != s->pending.end();) {
        Request &r = *s->reqs[*it];
        if (r.cancel) {
          rhpdhg_result res{};
          res.status = RHPDHG_STATUS_CANCELLED;
          finish_request(s, r, res);
          it = s->pending.erase(it);
          continue;
        }
        const int64_t nnz = r.row_ptr.back();
        rhpdhg_problem p = r.problem();
        bool admitted = false;
        if (nnz <= s->small_nnz && !r.params.adaptive_step && r.params.precision != 2) {
          int32_t slot = -1;
          const int rc = rhpdhg_batch_add(s->batch, &p, &r.params, &slot);
          if (rc == RHPDHG_OK) {
            r.where = 1;
            r.slot = slot;
            s->admitted_batched++;
            admitted = true;
          }
        } else {
          const int64_t need = single_lp_bytes(r);
          if (s->in_use + need <= s->budget) {
            rhpdhg_handle *h = nullptr;
            const int rc = rhpdhg_create(&p, &r.params, nullptr, &h);
            if (rc == RHPDHG_OK && rhpdhg_solve(h, 0) == RHPDHG_OK) {
              r.h = h;
              r.bytes = need;
              s->in_use += need;
              s->peak_in_use = std::max(s->peak_in_use, s->in_use);
              r.where = 2;
              s->admitted_single++;
              admitted = true;
            } else {
              if (h) rhpdhg_free(h);
              rhpdhg_result res{};
              res.status = RHPDHG_STATUS_NUMERICAL_ERROR;
              finish_request(s, r, res);
              it = s->pending.erase(it);
              continue;
            }
          }
        }
        if (admitted) {
          r.t_admit = Clock::now();
          it = s->pending.erase(it);
        } else {
          ++it;
        }
      }
      for (auto &kv : s->reqs) {
        if (kv.second->where == 1) batched_active = true;
        if (kv.second->where == 2) singles.push_back(kv.second.get());
      }
      if (!batched_active && singles.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    // ---- progress of the batched slots (one launch) ----
    if (batched_active) {
      rhpdhg_batch_step(s->batch, s->iters_per_step);
      s->steps++;
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    std::unique_lock<std::mutex> lk(s->mu);
    for (auto &kv : s->reqs) {
      Request &r = *kv.second;
      if (r.where == 1) {
        const int st = rhpdhg_batch_slot_status(s->batch, r.slot);
        if (st == RHPDHG_STATUS_RUNNING && !r.cancel) continue;
        rhpdhg_result res{};
        res.out_memory = RHPDHG_MEM_HOST;
        r.x.assign(r.n, 0.0);
        r.y.assign((size_t)r.m_eq + r.m_ineq, 0.0);
        r.cx.assign(r.n, 0.0);
        r.cy.assign((size_t)r.m_eq + r.m_ineq, 0.0);
        res.x = r.x.data();
        res.y = r.y.data();
        res.cert_x = r.cx.data();
        res.cert_y = r.cy.data();
        if (st == RHPDHG_STATUS_RUNNING) {
          res.status = RHPDHG_STATUS_CANCELLED;
        } else {
          rhpdhg_batch_poll(s->batch, r.slot, &res);
        }
        rhpdhg_batch_remove(s->batch, r.slot);
        r.slot = -1;
        finish_request(s, r, res);
      } else if (r.where == 2) {
        if (r.cancel) rhpdhg_cancel(r.h);
        rhpdhg_result res{};
        res.out_memory = RHPDHG_MEM_HOST;
        r.x.assign(r.n, 0.0);
        r.y.assign((size_t)r.m_eq + r.m_ineq, 0.0);
        r.cx.assign(r.n, 0.0);
        r.cy.assign((size_t)r.m_eq + r.m_ineq, 0.0);
        res.x = r.x.data();
        res.y = r.y.data();
        res.cert_x = r.cx.data();
        res.cert_y = r.cy.data();
        if (rhpdhg_poll(r.h, &res) == RHPDHG_BUSY) continue;
        rhpdhg_free(r.h);
        r.h = nullptr;
        s->in_use -= r.bytes;
        finish_request(s, r, res);
      }
    }
  }
}

}  // namespace

extern "C" {

int rhpdhg_server_create(int64_t budget_bytes, int64_t small_nnz, int32_t max_slots,
                         int32_t iters_per_step, rhpdhg_server **out) {
  if (!out || budget_bytes <= 0 || max_slots < 1 || iters_per_step < 1 || small_nnz < 0)
    return RHPDHG_ERR_INVALID_ARG;
  *out = nullptr;
  auto *s = new rhpdhg_server();
  cudaGetDevice(&s->dev);
  s->budget = budget_bytes;
  s->small_nnz = small_nnz;
  s->iters_per_step = iters_per_step;
  // the batched slots' arena: a quarter of the budget, at most enough for max_slots LPs of the
  // small-size limit
  rhpdhg_problem probe{};
  probe.m_eq = (int32_t)std::min<int64_t>(small_nnz / 5 + 1, INT32_MAX / 2);
  probe.n = (int32_t)std::min<int64_t>(small_nnz / 5 * 2 + 1, INT32_MAX / 2);
  probe.nnz = small_nnz;
  const int64_t per = rhpdhg_batch_bytes_needed(&probe, 1);
  s->arena_bytes = std::max<int64_t>(std::min<int64_t>(budget_bytes / 4, per * max_slots), 1 << 20);
  const int rc = rhpdhg_batch_create(max_slots, s->arena_bytes, nullptr, &s->batch);
  if (rc != RHPDHG_OK) {
    delete s;
    return rc;
  }
  s->in_use = s->arena_bytes;
  s->peak_in_use = s->in_use;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return RHPDHG_OK;
}

int rhpdhg_server_submit(rhpdhg_server *s, const rhpdhg_problem *lp, const rhpdhg_params *p,
                         int64_t *ticket) {
  if (!s || !lp || !ticket || lp->memory != RHPDHG_MEM_HOST || lp->n < 1 || lp->m_eq < 0 ||
      lp->m_ineq < 0 || lp->nnz < 0 || !lp->row_ptr)
    return RHPDHG_ERR_INVALID_ARG;
  auto r = std::make_unique<Request>();
  const int64_t m = (int64_t)lp->m_eq + lp->m_ineq;
  r->m_eq = lp->m_eq;
  r->m_ineq = lp->m_ineq;
  r->n = lp->n;
  r->obj_offset = lp->obj_offset;
  r->row_ptr.assign(lp->row_ptr, lp->row_ptr + m + 1);
  if (lp->nnz) {
    r->col_idx.assign(lp->col_idx, lp->col_idx + lp->nnz);
    r->val.assign(lp->val, lp->val + lp->nnz);
  }
  r->c.assign(lp->c, lp->c + lp->n);
  if (m) r->rhs.assign(lp->rhs, lp->rhs + m);
  r->l.assign(lp->l, lp->l + lp->n);
  r->u.assign(lp->u, lp->u + lp->n);
  if (p) r->params = *p;
  else rhpdhg_params_default(&r->params);
  r->params.x0 = nullptr;
  r->params.y0 = nullptr;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->pending.push_back(r->ticket);
  s->reqs[r->ticket] = std::move(r);
  s->cv.notify_one();
  return RHPDHG_OK;
}

int rhpdhg_server_poll(rhpdhg_server *s, int64_t ticket, rhpdhg_result *r, double *latency_s) {
  if (!s || !r) return RHPDHG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RHPDHG_ERR_INVALID_ARG;
  Request &q = *it->second;
  if (q.where != 3) return RHPDHG_BUSY;
  rhpdhg_result out = q.res;
  out.solve_seconds = std::chrono::duration<double>(q.t_done - q.t_admit).count();
  const int64_t m = (int64_t)q.m_eq + q.m_ineq;
  auto cp = [](double *dst, const std::vector<double> &src, int64_t cnt) {
    if (dst && cnt > 0 && (int64_t)src.size() >= cnt) std::memcpy(dst, src.data(), cnt * 8);
  };
  cp(r->x, q.x, q.n);
  cp(r->y, q.y, m);
  cp(r->cert_x, q.cx, q.n);
  cp(r->cert_y, q.cy, m);
  double *px = r->x, *py = r->y, *pcx = r->cert_x, *pcy = r->cert_y;
  *r = out;
  r->x = px;
  r->y = py;
  r->cert_x = pcx;
  r->cert_y = pcy;
  if (latency_s) *latency_s = std::chrono::duration<double>(q.t_done - q.t_submit).count();
  s->reqs.erase(it);
  return RHPDHG_OK;
}

int rhpdhg_server_cancel(rhpdhg_server *s, int64_t ticket) {
  if (!s) return RHPDHG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return RHPDHG_ERR_INVALID_ARG;
  it->second->cancel = true;
  s->cv.notify_one();
  return RHPDHG_OK;
}

int rhpdhg_server_stats(rhpdhg_server *s, int64_t *out) {
  if (!s || !out) return RHPDHG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t pend = (int64_t)s->pending.size(), batched = 0, single = 0;
  for (auto &kv : s->reqs) {
    if (kv.second->where == 1) batched++;
    if (kv.second->where == 2) single++;
  }
  out[0] = pend;
  out[1] = batched;
  out[2] = single;
  out[3] = s->completed;
  out[4] = s->in_use;
  out[5] = s->peak_in_use;
  out[6] = s->budget;
  out[7] = s->steps;
  out[8] = s->admitted_batched;
  out[9] = s->admitted_single;
  return RHPDHG_OK;
}

void rhpdhg_server_free(rhpdhg_server *s) {
  if (!s) return;
  s->stop = true;
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->reqs)
    if (kv.second->h) rhpdhg_free(kv.second->h);
  rhpdhg_batch_free(s->batch);
  delete s;
}

}  // extern "C"
