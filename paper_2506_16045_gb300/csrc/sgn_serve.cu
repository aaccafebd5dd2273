// Serving: continuous batching of SGN constraint solves and runs on one GPU.
//
// A worker thread owns a stream and a private sgn_ctx.  Submissions copy their arrays to
// the device and queue; the worker admits queued requests in arrival order while their
// memory footprint fits the budget (a later, smaller request may pass a blocked larger
// one), then repeatedly:
//   * runs all admitted 1d solves as one batched PCG launch group;
//   * advances all admitted 1d RK4 runs together by a chunk of steps through one batched
//     layout (per-instance dt), gathering and scattering their device state around it;
//   * advances 2d and multistep runs, and runs 2d solves, per request;
//   * completes finished requests and frees their workspace.
// RK4 is a one-step method and every instance of a batched launch is computed by its own
// CTAs, so a request's result does not depend on which requests shared its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/sgn.h"
#include "sgn_internal.h"

namespace sgn {
sgn_status state_attach(sgn_state* st, cudaStream_t s);
}

namespace {

constexpr int kChunk = 16;           // RUN steps per scheduling round

struct Req {
  uint64_t ticket = 0;
  sgn_request q{};
  int d = 1;
  long long N = 0;
  size_t footprint = 0;
  // device arrays owned by the request
  double* eta = nullptr;
  double* u = nullptr;                // u (RUN) or the solution x (SOLVE)
  double* b = nullptr;                // SOLVE right-hand side
  double* h = nullptr;
  double* U = nullptr;
  double* gh = nullptr;
  // per-request objects (2d / multistep runs, 2d solves)
  sgn_layout* lay = nullptr;
  sgn_state* st = nullptr;
  int remaining = 0;
  bool admitted = false, done = false;
  sgn_status status = SGN_OK;
  sgn_pcg_info info{};
  long long iters = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace

struct sgn_server {
  int device = 0;
  sgn_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t copy = nullptr;
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> all;
  uint64_t next = 1;
  bool stop = false;
  std::thread worker;
  // cached batch objects for 1d RK4 runs
  std::vector<uint64_t> run_members;
  sgn_layout* run_lay = nullptr;
  sgn_state* run_st = nullptr;
  double* pk = nullptr;               // packed eta, U, u, h, gh of the RK4 batch (5 x cap)
  long long pk_cap = 0;
  double* pks = nullptr;              // packed eta, b, x, gh of a solve batch
  long long pks_cap = 0;
  std::map<std::pair<int, double>, sgn_layout*> one1d;   // single-instance 1d layouts
};

namespace {

size_t footprint_of(int d, long long N) {
  const size_t io = (size_t)(2 + 3 * d) * 8 * N;          // eta, h, u/b, U, gradh
  const size_t work = d == 1 ? (size_t)260 * N : (size_t)816 * N;
  const size_t big = (d == 1 && N > 8192) ? (size_t)16 * N : 0;   // global transform buffer
  return io + work + big + (1 << 16);
}

void free_req_work(Req* r) {
  if (r->st) sgn_state_free(r->st);
  if (r->lay) sgn_layout_destroy(r->lay);
  r->st = nullptr;
  r->lay = nullptr;
  cudaFree(r->h);
  cudaFree(r->gh);
  cudaFree(r->b);
  r->h = r->gh = r->b = nullptr;
}

void free_req_all(Req* r) {
  free_req_work(r);
  cudaFree(r->eta);
  cudaFree(r->u);
  cudaFree(r->U);
  delete r;
}

sgn_layout* one_layout(sgn_server* S, const sgn_grid& g) {
  auto key = std::make_pair(g.nx, g.Lx);
  auto it = S->one1d.find(key);
  if (it != S->one1d.end()) return it->second;
  sgn_layout* lay = nullptr;
  if (sgn_layout_create(S->ctx, 1, &g, &lay) != SGN_OK) return nullptr;
  S->one1d[key] = lay;
  return lay;
}

void finish(sgn_server* S, Req* r, sgn_status st) {
  const double t = now_s();
  free_req_work(r);
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->t_done = t;
  r->done = true;
  S->used -= r->footprint;
}

bool is_batched_run(const Req* r) {
  return r->q.kind == SGN_REQ_RUN && r->d == 1 && r->q.scheme == SGN_SCHEME_RK4;
}

// Initialise an admitted request on the device.
sgn_status start(sgn_server* S, Req* r) {
  const sgn_stream s = S->stream;
  if (r->q.kind == SGN_REQ_RUN && is_batched_run(r)) {
    sgn_layout* lay = one_layout(S, r->q.grid);
    if (!lay) return SGN_ERR_NOMEM;
    sgn_status e = sgn_spectral_grad(S->ctx, lay, r->h, r->gh, s);
    if (e) return e;
    return sgn_apply_operator(S->ctx, lay, r->eta, r->gh, r->u, r->U, s);
  }
  if (r->q.kind == SGN_REQ_RUN) {
    sgn_status e = sgn_layout_create(S->ctx, 1, &r->q.grid, &r->lay);
    if (e) return e;
    if ((e = sgn_state_create(S->ctx, r->lay, r->eta, r->U, r->u, r->h, r->gh, &r->st))) return e;
    return sgn_state_init(r->st, s);
  }
  // SOLVE: grad h now (2d solves also get their layout here)
  if (r->d == 2) {
    sgn_status e = sgn_layout_create(S->ctx, 1, &r->q.grid, &r->lay);
    if (e) return e;
    return sgn_spectral_grad(S->ctx, r->lay, r->h, r->gh, s);
  }
  sgn_layout* lay = one_layout(S, r->q.grid);
  if (!lay) return SGN_ERR_NOMEM;
  return sgn_spectral_grad(S->ctx, lay, r->h, r->gh, s);
}

// grow-only packed buffer of 5 P doubles
sgn_status ensure_pack(double** buf, long long* cap, long long P) {
  if (P <= *cap) return SGN_OK;
  cudaFree(*buf);
  *buf = nullptr;
  if (cudaMalloc(buf, sizeof(double) * 5 * (size_t)P) != cudaSuccess) {
    cudaGetLastError();
    *cap = 0;
    return SGN_ERR_NOMEM;
  }
  *cap = P;
  return SGN_OK;
}

// All admitted 1d solves as one batched PCG (grouped by options).
void run_solves_1d(sgn_server* S, std::vector<Req*>& v) {
  if (v.empty()) return;
  std::vector<sgn_grid> grids;
  for (Req* r : v) grids.push_back(r->q.grid);
  sgn_layout* lay = nullptr;
  sgn_status e = sgn_layout_create(S->ctx, (int)v.size(), grids.data(), &lay);
  if (e) {
    for (Req* r : v) finish(S, r, e);
    return;
  }
  std::vector<long long> off(v.size() + 1);
  sgn_layout_offsets(lay, off.data());
  const long long P = off.back();
  if ((e = ensure_pack(&S->pks, &S->pks_cap, P))) {
    sgn_layout_destroy(lay);
    for (Req* r : v) finish(S, r, e);
    return;
  }
  double *pe = S->pks, *pb = S->pks + P, *px = S->pks + 2 * P, *pg = S->pks + 3 * P;
  for (size_t i = 0; i < v.size(); ++i) {
    const size_t bytes = sizeof(double) * (size_t)v[i]->N;
    cudaMemcpyAsync(pe + off[i], v[i]->eta, bytes, cudaMemcpyDeviceToDevice, S->stream);
    cudaMemcpyAsync(pb + off[i], v[i]->b, bytes, cudaMemcpyDeviceToDevice, S->stream);
    cudaMemcpyAsync(pg + off[i], v[i]->gh, bytes, cudaMemcpyDeviceToDevice, S->stream);
  }
  cudaMemsetAsync(px, 0, sizeof(double) * P, S->stream);
  const sgn_opts& o = v[0]->q.opts;
  std::vector<sgn_pcg_info> info(v.size());
  e = sgn_pcg(S->ctx, lay, pe, pg, nullptr, pb, px, o.rtol, o.maxit, o.prec, info.data(),
              S->stream);
  for (size_t i = 0; i < v.size(); ++i)
    cudaMemcpyAsync(v[i]->u, px + off[i], sizeof(double) * (size_t)v[i]->N,
                    cudaMemcpyDeviceToDevice, S->stream);
  cudaStreamSynchronize(S->stream);
  sgn_layout_destroy(lay);
  for (size_t i = 0; i < v.size(); ++i) {
    v[i]->info = info[i];
    finish(S, v[i], e == SGN_ERR_CUDA ? e : (sgn_status)info[i].status);
  }
}

// Advance all admitted 1d RK4 runs together by K steps.
void run_batch_rk4(sgn_server* S, std::vector<Req*>& v) {
  if (v.empty()) return;
  int K = kChunk;
  for (Req* r : v) K = std::min(K, r->remaining);
  std::vector<uint64_t> members;
  for (Req* r : v) members.push_back(r->ticket);
  sgn_status e = SGN_OK;
  if (members != S->run_members) {
    if (S->run_st) sgn_state_free(S->run_st);
    if (S->run_lay) sgn_layout_destroy(S->run_lay);
    S->run_st = nullptr;
    S->run_lay = nullptr;
    S->run_members.clear();
    std::vector<sgn_grid> grids;
    for (Req* r : v) grids.push_back(r->q.grid);
    e = sgn_layout_create(S->ctx, (int)v.size(), grids.data(), &S->run_lay);
    long long P = e ? 0 : sgn_layout_points(S->run_lay);
    if (!e) e = ensure_pack(&S->pk, &S->pk_cap, P);
    if (!e)
      e = sgn_state_create(S->ctx, S->run_lay, S->pk, S->pk + P, S->pk + 2 * P, S->pk + 3 * P,
                           S->pk + 4 * P, &S->run_st);
    if (e) {
      for (Req* r : v) finish(S, r, e);
      return;
    }
    S->run_members = members;
  }
  sgn_layout* lay = S->run_lay;
  std::vector<long long> off(v.size() + 1);
  sgn_layout_offsets(lay, off.data());
  const long long P = off.back();
  double* F[5] = {S->pk, S->pk + P, S->pk + 2 * P, S->pk + 3 * P, S->pk + 4 * P};
  for (size_t i = 0; i < v.size(); ++i) {
    double* src[5] = {v[i]->eta, v[i]->U, v[i]->u, v[i]->h, v[i]->gh};
    for (int f = 0; f < 5; ++f)
      cudaMemcpyAsync(F[f] + off[i], src[f], sizeof(double) * (size_t)v[i]->N,
                      cudaMemcpyDeviceToDevice, S->stream);
  }
  std::vector<double> dts;
  for (Req* r : v) dts.push_back(r->q.dt);
  e = sgn::state_attach(S->run_st, S->stream);
  const sgn_opts& o = v[0]->q.opts;
  if (!e) e = sgn_step_rk4(S->run_st, dts.data(), K, &o, S->stream);
  for (size_t i = 0; i < v.size(); ++i) {
    double* dst[3] = {v[i]->eta, v[i]->U, v[i]->u};
    for (int f = 0; f < 3; ++f)
      cudaMemcpyAsync(dst[f], F[f] + off[i], sizeof(double) * (size_t)v[i]->N,
                      cudaMemcpyDeviceToDevice, S->stream);
  }
  sgn_state_stats stt{};
  if (!e) e = sgn_state_get_stats(S->run_st, &stt);
  cudaStreamSynchronize(S->stream);
  for (Req* r : v) {
    r->remaining -= K;
    r->iters += stt.iterations / (long long)v.size();   // shared launches: mean per request
    if (e || stt.status != SGN_OK) {
      finish(S, r, e ? e : (sgn_status)stt.status);
    } else if (r->remaining <= 0) {
      r->info.iters = (int)r->iters;
      finish(S, r, SGN_OK);
    }
  }
}

void run_single(sgn_server* S, Req* r) {
  sgn_status e = SGN_OK;
  if (r->q.kind == SGN_REQ_SOLVE) {
    cudaMemsetAsync(r->u, 0, sizeof(double) * r->d * (size_t)r->N, S->stream);
    sgn_pcg_info info{};
    const sgn_opts& o = r->q.opts;
    e = sgn_pcg(S->ctx, r->lay, r->eta, r->gh, nullptr, r->b, r->u, o.rtol, o.maxit, o.prec,
                &info, S->stream);
    r->info = info;
    finish(S, r, e == SGN_ERR_CUDA ? e : (sgn_status)info.status);
    return;
  }
  const int K = std::min(kChunk, r->remaining);
  const sgn_opts& o = r->q.opts;
  const double dt = r->q.dt;
  switch (r->q.scheme) {
    case SGN_SCHEME_RK4: e = sgn_step_rk4(r->st, &dt, K, &o, S->stream); break;
    case SGN_SCHEME_LINIMP: e = sgn_step_linimp(r->st, &dt, K, &o, S->stream); break;
    default: e = sgn_step_abk(r->st, (int)r->q.scheme, &dt, K, &o, S->stream); break;
  }
  sgn_state_stats stt{};
  if (!e) e = sgn_state_get_stats(r->st, &stt);
  r->remaining -= K;
  if (e || stt.status != SGN_OK) {
    finish(S, r, e ? e : (sgn_status)stt.status);
  } else if (r->remaining <= 0) {
    r->info.iters = (int)stt.iterations;
    finish(S, r, SGN_OK);
  }
}

void worker_main(sgn_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Req*> admit_now;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::milliseconds(2),
                     [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
      if (S->stop && S->pending.empty() && S->active.empty()) break;
      for (auto it = S->pending.begin(); it != S->pending.end();) {
        Req* r = *it;
        if (S->used + r->footprint <= S->budget) {
          S->used += r->footprint;
          r->admitted = true;
          r->t_admit = now_s();
          admit_now.push_back(r);
          it = S->pending.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (Req* r : admit_now) {
      sgn_status e = start(S, r);
      if (e) {
        finish(S, r, e);
        continue;
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.push_back(r);
    }
    std::vector<Req*> act;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      act = S->active;
    }
    if (act.empty()) continue;
    std::vector<Req*> solves1d, runs1d, singles;
    for (Req* r : act) {
      if (r->done) continue;
      if (r->q.kind == SGN_REQ_SOLVE && r->d == 1) solves1d.push_back(r);
      else if (is_batched_run(r)) runs1d.push_back(r);
      else singles.push_back(r);
    }
    // 1d solves grouped by identical options, batched
    while (!solves1d.empty()) {
      const sgn_opts o = solves1d[0]->q.opts;
      std::vector<Req*> grp, rest;
      for (Req* r : solves1d)
        (memcmp(&r->q.opts, &o, sizeof(o)) == 0 ? grp : rest).push_back(r);
      run_solves_1d(S, grp);
      solves1d.swap(rest);
    }
    while (!runs1d.empty()) {
      const sgn_opts o = runs1d[0]->q.opts;
      std::vector<Req*> grp, rest;
      for (Req* r : runs1d) (memcmp(&r->q.opts, &o, sizeof(o)) == 0 ? grp : rest).push_back(r);
      run_batch_rk4(S, grp);
      runs1d.swap(rest);
    }
    for (Req* r : singles) run_single(S, r);
    std::lock_guard<std::mutex> lk(S->mu);
    S->active.erase(std::remove_if(S->active.begin(), S->active.end(),
                                   [](Req* r) { return r->done; }),
                    S->active.end());
  }
}

}  // namespace

extern "C" double sgn_clock(void) { return now_s(); }

extern "C" sgn_status sgn_server_create(sgn_ctx* ctx, double budget_fraction, sgn_server** out) {
  if (!ctx || !out) return SGN_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  sgn_server* S = new (std::nothrow) sgn_server();
  if (!S) return SGN_ERR_NOMEM;
  S->device = dev;
  sgn_status e = sgn_create(&S->ctx, dev, 0);
  if (e) {
    delete S;
    return e;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    sgn_destroy(S->ctx);
    delete S;
    return SGN_ERR_CUDA;
  }
  const double f = budget_fraction > 0.0 ? budget_fraction : 0.8;
  S->budget = (size_t)(f * (double)tot);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return SGN_OK;
}

extern "C" sgn_status sgn_batch_submit(sgn_server* S, const sgn_request* q, uint64_t* ticket) {
  if (!S || !q || !ticket || !q->eta || !q->u_or_b || !q->h) return SGN_ERR_INVALID_ARG;
  const sgn_grid& g = q->grid;
  const int d = g.dim;
  if (d == 1) {
    if (g.ny != 1 || !pow2_in(g.nx, 8, 16384)) return SGN_ERR_UNSUPPORTED_SIZE;
  } else if (d == 2) {
    if (!pow2_in(g.nx, 8, 1024) || !pow2_in(g.ny, 8, 1024)) return SGN_ERR_UNSUPPORTED_SIZE;
  } else {
    return SGN_ERR_INVALID_ARG;
  }
  if (!(g.Lx > 0.0) || (d == 2 && !(g.Ly > 0.0))) return SGN_ERR_INVALID_ARG;
  if (q->kind == SGN_REQ_RUN &&
      (!(q->dt > 0.0) || q->nsteps < 0 ||
       (q->scheme != SGN_SCHEME_RK4 && q->scheme != SGN_SCHEME_LINIMP &&
        (q->scheme < SGN_SCHEME_AB2 || q->scheme > SGN_SCHEME_AB4))))
    return SGN_ERR_INVALID_ARG;
  if (q->kind != SGN_REQ_RUN && q->kind != SGN_REQ_SOLVE) return SGN_ERR_INVALID_ARG;
  if (!(q->opts.rtol > 0.0) || q->opts.maxit <= 0) return SGN_ERR_INVALID_ARG;
  Req* r = new (std::nothrow) Req();
  if (!r) return SGN_ERR_NOMEM;
  r->q = *q;
  r->d = d;
  r->N = (long long)g.nx * g.ny;
  r->footprint = footprint_of(d, r->N);
  if (r->footprint > S->budget) {
    delete r;
    return SGN_ERR_REJECTED;
  }
  r->remaining = q->kind == SGN_REQ_RUN ? q->nsteps : 0;
  r->t_submit = now_s();
  const size_t sN = sizeof(double) * (size_t)r->N;
  cudaSetDevice(S->device);
  bool ok = cudaMalloc(&r->eta, sN) == cudaSuccess && cudaMalloc(&r->h, sN) == cudaSuccess &&
            cudaMalloc(&r->u, d * sN) == cudaSuccess && cudaMalloc(&r->gh, d * sN) == cudaSuccess &&
            cudaMalloc(&r->U, d * sN) == cudaSuccess;
  if (ok && q->kind == SGN_REQ_SOLVE) ok = cudaMalloc(&r->b, d * sN) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_req_all(r);
    return SGN_ERR_NOMEM;
  }
  const cudaMemcpyKind k = q->host_memory ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyAsync(r->eta, q->eta, sN, k, S->copy);
  cudaMemcpyAsync(r->h, q->h, sN, k, S->copy);
  cudaMemcpyAsync(q->kind == SGN_REQ_SOLVE ? r->b : r->u, q->u_or_b, d * sN, k, S->copy);
  if (cudaStreamSynchronize(S->copy) != cudaSuccess) {
    cudaGetLastError();
    free_req_all(r);
    return SGN_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next++;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
  }
  S->cv.notify_one();
  *ticket = r->ticket;
  return SGN_OK;
}

extern "C" sgn_status sgn_batch_poll(sgn_server* S, uint64_t ticket, sgn_result* out) {
  if (!S || !out) return SGN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return SGN_ERR_INVALID_ARG;
  Req* r = it->second;
  if (!r->done) return SGN_ERR_PENDING;
  out->status = r->status;
  const bool run = r->q.kind == SGN_REQ_RUN;
  out->eta = run ? r->eta : nullptr;
  out->u = r->u;
  out->U = run ? r->U : nullptr;
  out->info = r->info;
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
  return r->status;
}

extern "C" sgn_status sgn_result_release(sgn_server* S, uint64_t ticket) {
  if (!S) return SGN_ERR_INVALID_ARG;
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SGN_ERR_INVALID_ARG;
    if (!it->second->done) return SGN_ERR_PENDING;
    r = it->second;
    S->all.erase(it);
  }
  cudaSetDevice(S->device);
  free_req_all(r);
  return SGN_OK;
}

extern "C" void sgn_server_destroy(sgn_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_one();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  for (auto& kv : S->all) free_req_all(kv.second);
  if (S->run_st) sgn_state_free(S->run_st);
  if (S->run_lay) sgn_layout_destroy(S->run_lay);
  for (auto& kv : S->one1d) sgn_layout_destroy(kv.second);
  cudaFree(S->pk);
  cudaFree(S->pks);
  cudaStreamDestroy(S->stream);
  cudaStreamDestroy(S->copy);
  sgn_destroy(S->ctx);
  delete S;
}
