// Serving: continuous batching of SGN constraint solves and runs on one GPU.
//
// A worker thread owns a private sgn_ctx and a set of CUDA streams ("lanes").  Submissions
// copy their arrays to the device and queue; the worker admits queued requests in arrival
// order while their memory footprint fits the budget (a later, smaller request may pass a
// blocked larger one) and keeps every admitted request moving without waiting on the GPU:
//   * admitted 1d solves, grouped by options, run as one batched PCG per group on a
//     high-priority solve lane, their reports written to device memory (sgn_pcg_async);
//   * admitted 1d RK4 runs advance together, a chunk of steps at a time, through one batched
//     layout (per-instance dt) on the batch lane, gathering and scattering their device
//     state around each chunk;
//   * 1d multistep runs (AB2-4, SBDF2) advance chunk by chunk on their own lanes;
//   * 2d solves and 2d runs share the 2d lane, which has the highest priority: their
//     inner solves are cooperative persistent launches, which must not wait on one another;
//   * each piece of work ends with an event; the worker polls the events, completes the
//     finished requests and issues the next chunk, so the lanes' work overlaps on the device.
// Work that frees device memory (cudaFree waits for the whole device) is deferred until no
// lane is busy, or until the deferred bytes pass a threshold.
// RK4 is a one-step method and every instance of a batched launch is computed by its own
// CTAs, and a 2d or multistep request runs on its own layout and state, so a request's
// result does not depend on which requests ran beside it.
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
#include "sgn_2d.h"
#include "sgn_internal.h"

namespace sgn {
sgn_status state_attach(sgn_state* st, cudaStream_t s);
double* state_rk4_prev(sgn_state* st);
double* state_rk4_last(sgn_state* st);
}

namespace {

constexpr int kChunk = 16;           // RUN steps per scheduling round
constexpr int kSolveLanes = 2;       // high-priority lanes of the 1d solve groups
constexpr size_t kReapBytes = (size_t)2 << 30;   // deferred frees forced past this many bytes

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
  double* hist = nullptr;             // batched 1d RK4 runs: the RK4 history (u_prev, u_last)
  // per-request objects (2d / multistep runs, 2d solves)
  sgn_layout* lay = nullptr;
  sgn_state* st = nullptr;
  cudaEvent_t ready = nullptr;        // the request's set-up work (grad h, U = G u) is done
  cudaStream_t own = nullptr;         // 1d multistep runs: their own lane
  bool busy = false;                  // a job of this request is in flight
  double last_issue = 0.0;            // when its last job was issued (2d lane turns)
  int remaining = 0;
  bool admitted = false, done = false;
  // ownership after `done` (under the server's mutex): the worker frees the request's
  // working memory (reaped); the client gives up its result (released).  Whichever comes
  // second deletes the request.
  bool reaped = false, released = false;
  sgn_status status = SGN_OK;
  sgn_pcg_info info{};
  long long iters = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// One piece of issued work: the requests it serves, its lane and its completion event.
enum JobKind { JOB_SOLVES_1D = 0, JOB_RUN_BATCH = 1, JOB_SINGLE = 2 };
struct Job {
  JobKind kind;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<Req*> reqs;
  sgn_layout* lay = nullptr;          // a solve group's layout
  int info_at = -1, info_n = 0;       // slots of the report pool
  int K = 0;                          // steps of a run chunk
  sgn_status err = SGN_OK;            // an issue-time failure
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
  cudaStream_t stream = nullptr;      // set-up work of admitted requests
  cudaStream_t copy = nullptr;        // submissions' input copies
  cudaStream_t lane_solve[kSolveLanes] = {};
  cudaStream_t lane_batch = nullptr;
  cudaStream_t lane_2d = nullptr;
  int prio_lo = 0, prio_hi = 0;       // stream priority range (hi: the greatest)
  int next_solve_lane = 0;
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> all;
  uint64_t next = 1;
  bool stop = false;
  std::thread worker;
  std::vector<Job*> inflight;
  std::vector<cudaEvent_t> events;    // completed jobs' events, reused
  // reports of solve jobs: device slots and their pinned host copies
  sgn_pcg_info* info_dev = nullptr;
  sgn_pcg_info* info_host = nullptr;
  std::vector<char> info_used;
  // deferred frees (cudaFree waits for the device)
  std::vector<Req*> reap_reqs;
  std::vector<sgn_layout*> reap_lays;
  std::vector<sgn_state*> reap_states;
  size_t reap_bytes = 0;
  // cached batch objects for 1d RK4 runs
  std::vector<uint64_t> run_members;
  bool batch_busy = false;
  sgn_layout* run_lay = nullptr;
  sgn_state* run_st = nullptr;
  double* pk = nullptr;               // packed eta, U, u, h, gh of the RK4 batch (5 x cap)
  long long pk_cap = 0;
  std::map<std::pair<int, double>, sgn_layout*> one1d;   // single-instance 1d layouts
};

namespace {

constexpr int kInfoSlots = 8192;

size_t footprint_of(int d, long long N) {
  const size_t io = (size_t)(2 + 3 * d) * 8 * N + (d == 1 ? 16 * N : 0);   // + RK4 history
  const size_t work = d == 1 ? (size_t)260 * N : (size_t)816 * N;
  const size_t big = (d == 1 && N > 6144) ? (size_t)32 * N : 0;   // global transform buffers
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
  cudaFree(r->hist);
  r->h = r->gh = r->b = r->hist = nullptr;
  if (r->ready) cudaEventDestroy(r->ready);
  r->ready = nullptr;
  if (r->own) cudaStreamDestroy(r->own);
  r->own = nullptr;
}

void free_req_all(Req* r) {
  free_req_work(r);
  cudaFree(r->eta);
  cudaFree(r->u);
  cudaFree(r->U);
  delete r;
}

// Frees deferred work, which waits for the device: only when no lane is busy, unless the
// deferred memory has grown past kReapBytes.  A request the client has already released
// is deleted here; otherwise sgn_result_release deletes it later.
void reap(sgn_server* S, bool force) {
  if (S->reap_reqs.empty() && S->reap_lays.empty() && S->reap_states.empty()) return;
  if (!force && !S->inflight.empty() && S->reap_bytes < kReapBytes) return;
  for (Req* r : S->reap_reqs) {
    free_req_work(r);
    bool gone;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->reaped = true;
      gone = r->released;
    }
    if (gone) free_req_all(r);
  }
  for (sgn_state* st : S->reap_states) sgn_state_free(st);
  for (sgn_layout* l : S->reap_lays) sgn_layout_destroy(l);
  S->reap_reqs.clear();
  S->reap_states.clear();
  S->reap_lays.clear();
  S->reap_bytes = 0;
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

// The request is finished: publish its result; its working memory is freed later.
void finish(sgn_server* S, Req* r, sgn_status st) {
  const double t = now_s();
  S->reap_reqs.push_back(r);
  S->reap_bytes += r->footprint;
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->t_done = t;
  r->done = true;
  r->busy = false;
  S->used -= r->footprint;
}

bool is_batched_run(const Req* r) {
  return r->q.kind == SGN_REQ_RUN && r->d == 1 && r->q.scheme == SGN_SCHEME_RK4;
}

cudaEvent_t take_event(sgn_server* S) {
  if (!S->events.empty()) {
    cudaEvent_t e = S->events.back();
    S->events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

int take_info(sgn_server* S, int n) {
  for (int i = 0; i + n <= kInfoSlots; ++i) {
    int j = 0;
    while (j < n && !S->info_used[i + j]) ++j;
    if (j == n) {
      for (int k = 0; k < n; ++k) S->info_used[i + k] = 1;
      return i;
    }
    i += j;
  }
  return -1;
}

void give_info(sgn_server* S, int at, int n) {
  for (int k = 0; k < n; ++k) S->info_used[at + k] = 0;
}

// Initialise an admitted request on the device (the set-up stream); records r->ready.
sgn_status start(sgn_server* S, Req* r) {
  const sgn_stream s = S->stream;
  sgn_status e = SGN_OK;
  if (r->q.kind == SGN_REQ_RUN && is_batched_run(r)) {
    sgn_layout* lay = one_layout(S, r->q.grid);
    if (!lay) return SGN_ERR_NOMEM;
    // the request's own RK4 history travels with it through the batched state, so its
    // result does not depend on the requests beside it (no history yet: NaN)
    if (cudaMalloc(&r->hist, sizeof(double) * 2 * (size_t)r->N) != cudaSuccess ||
        cudaMemsetAsync(r->hist + r->N, 0xff, sizeof(double) * (size_t)r->N, S->stream) !=
            cudaSuccess) {
      cudaGetLastError();
      return SGN_ERR_NOMEM;
    }
    e = sgn_spectral_grad(S->ctx, lay, r->h, r->gh, s);
    if (!e) e = sgn_apply_operator(S->ctx, lay, r->eta, r->gh, r->u, r->U, s);
  } else if (r->q.kind == SGN_REQ_RUN) {
    e = sgn_layout_create(S->ctx, 1, &r->q.grid, &r->lay);
    if (!e) e = sgn_state_create(S->ctx, r->lay, r->eta, r->U, r->u, r->h, r->gh, &r->st);
    if (!e) e = sgn_state_init(r->st, s);
  } else if (r->d == 2) {
    // SOLVE: grad h now (2d solves also get their layout here)
    e = sgn_layout_create(S->ctx, 1, &r->q.grid, &r->lay);
    if (!e) e = sgn_spectral_grad(S->ctx, r->lay, r->h, r->gh, s);
  } else {
    sgn_layout* lay = one_layout(S, r->q.grid);
    if (!lay) return SGN_ERR_NOMEM;
    e = sgn_spectral_grad(S->ctx, lay, r->h, r->gh, s);
  }
  if (e) return e;
  if (!(r->ready = take_event(S)) || cudaEventRecord(r->ready, S->stream) != cudaSuccess) {
    cudaGetLastError();
    return SGN_ERR_CUDA;
  }
  return SGN_OK;
}

void wait_ready(cudaStream_t s, const std::vector<Req*>& v) {
  for (Req* r : v)
    if (r->ready) cudaStreamWaitEvent(s, r->ready, 0);
}

// Ends an issued job with its event and puts it in flight (or fails its requests).
void launch_job(sgn_server* S, Job* J) {
  if (!J->err) {
    J->ev = take_event(S);
    if (!J->ev || cudaEventRecord(J->ev, J->s) != cudaSuccess) {
      cudaGetLastError();
      J->err = SGN_ERR_CUDA;
    }
  }
  for (Req* r : J->reqs) r->busy = true;
  S->inflight.push_back(J);
}

// All given 1d solves (one option set) as one batched PCG with device-side reports.
void issue_solves_1d(sgn_server* S, std::vector<Req*>& v) {
  Job* J = new Job();
  J->kind = JOB_SOLVES_1D;
  J->reqs = v;
  J->s = S->lane_solve[S->next_solve_lane];
  S->next_solve_lane = (S->next_solve_lane + 1) % kSolveLanes;
  std::vector<sgn_grid> grids;
  for (Req* r : v) grids.push_back(r->q.grid);
  sgn_status e = sgn_layout_create(S->ctx, (int)v.size(), grids.data(), &J->lay);
  if (!e && (J->info_at = take_info(S, (int)v.size())) < 0) e = SGN_ERR_NOMEM;
  J->info_n = (int)v.size();
  double* pk = nullptr;
  long long P = 0;
  std::vector<long long> off(v.size() + 1);
  if (!e) {
    sgn_layout_offsets(J->lay, off.data());
    P = off.back();
    // the packed arrays of the group live with its layout (stream-ordered allocation)
    if (cudaMallocAsync(reinterpret_cast<void**>(&pk), sizeof(double) * 4 * (size_t)P, J->s) !=
        cudaSuccess) {
      cudaGetLastError();
      e = SGN_ERR_NOMEM;
    }
  }
  if (!e) {
    wait_ready(J->s, v);
    double *pe = pk, *pb = pk + P, *px = pk + 2 * P, *pg = pk + 3 * P;
    for (size_t i = 0; i < v.size(); ++i) {
      const size_t bytes = sizeof(double) * (size_t)v[i]->N;
      cudaMemcpyAsync(pe + off[i], v[i]->eta, bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(pb + off[i], v[i]->b, bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(pg + off[i], v[i]->gh, bytes, cudaMemcpyDeviceToDevice, J->s);
    }
    cudaMemsetAsync(px, 0, sizeof(double) * P, J->s);
    const sgn_opts& o = v[0]->q.opts;
    e = sgn_pcg_async(S->ctx, J->lay, pe, pg, pb, px, o.rtol, o.maxit, o.prec,
                      S->info_dev + J->info_at, J->s);
    for (size_t i = 0; i < v.size(); ++i)
      cudaMemcpyAsync(v[i]->u, px + off[i], sizeof(double) * (size_t)v[i]->N,
                      cudaMemcpyDeviceToDevice, J->s);
    cudaMemcpyAsync(S->info_host + J->info_at, S->info_dev + J->info_at,
                    sizeof(sgn_pcg_info) * v.size(), cudaMemcpyDeviceToHost, J->s);
    cudaFreeAsync(pk, J->s);
    if (cudaGetLastError() != cudaSuccess && !e) e = SGN_ERR_CUDA;
  }
  J->err = e;
  launch_job(S, J);
}

// The next chunk of all given 1d RK4 runs (one option set), on the batch lane.
void issue_run_batch(sgn_server* S, std::vector<Req*>& v) {
  Job* J = new Job();
  J->kind = JOB_RUN_BATCH;
  J->reqs = v;
  J->s = S->lane_batch;
  int K = kChunk;
  for (Req* r : v) K = std::min(K, r->remaining);
  J->K = K;
  std::vector<uint64_t> members;
  for (Req* r : v) members.push_back(r->ticket);
  sgn_status e = SGN_OK;
  if (members != S->run_members) {
    if (S->run_st) S->reap_states.push_back(S->run_st);
    if (S->run_lay) S->reap_lays.push_back(S->run_lay);
    S->run_st = nullptr;
    S->run_lay = nullptr;
    S->run_members.clear();
    std::vector<sgn_grid> grids;
    for (Req* r : v) grids.push_back(r->q.grid);
    e = sgn_layout_create(S->ctx, (int)v.size(), grids.data(), &S->run_lay);
    long long P = e ? 0 : sgn_layout_points(S->run_lay);
    if (!e && P > S->pk_cap) {
      // the packed buffer may still be read by an earlier chunk on this lane: free it in order
      if (S->pk) cudaFreeAsync(S->pk, J->s);
      S->pk = nullptr;
      S->pk_cap = 0;
      if (cudaMallocAsync(reinterpret_cast<void**>(&S->pk), sizeof(double) * 5 * (size_t)P,
                          J->s) != cudaSuccess) {
        cudaGetLastError();
        e = SGN_ERR_NOMEM;
      } else {
        S->pk_cap = P;
      }
    }
    if (!e)
      e = sgn_state_create(S->ctx, S->run_lay, S->pk, S->pk + P, S->pk + 2 * P, S->pk + 3 * P,
                           S->pk + 4 * P, &S->run_st);
    if (!e) S->run_members = members;
  }
  if (!e) {
    sgn_layout* lay = S->run_lay;
    std::vector<long long> off(v.size() + 1);
    sgn_layout_offsets(lay, off.data());
    const long long P = off.back();
    double* F[5] = {S->pk, S->pk + P, S->pk + 2 * P, S->pk + 3 * P, S->pk + 4 * P};
    wait_ready(J->s, v);
    double* Hp = sgn::state_rk4_prev(S->run_st);
    double* Hl = sgn::state_rk4_last(S->run_st);
    for (size_t i = 0; i < v.size(); ++i) {
      double* src[5] = {v[i]->eta, v[i]->U, v[i]->u, v[i]->h, v[i]->gh};
      const size_t bytes = sizeof(double) * (size_t)v[i]->N;
      for (int f = 0; f < 5; ++f)
        cudaMemcpyAsync(F[f] + off[i], src[f], bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(Hp + off[i], v[i]->hist, bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(Hl + off[i], v[i]->hist + v[i]->N, bytes, cudaMemcpyDeviceToDevice, J->s);
    }
    std::vector<double> dts;
    for (Req* r : v) dts.push_back(r->q.dt);
    e = sgn::state_attach(S->run_st, J->s);
    const sgn_opts& o = v[0]->q.opts;
    if (!e) e = sgn_step_rk4(S->run_st, dts.data(), K, &o, J->s);
    for (size_t i = 0; i < v.size(); ++i) {
      double* dst[3] = {v[i]->eta, v[i]->U, v[i]->u};
      const size_t bytes = sizeof(double) * (size_t)v[i]->N;
      for (int f = 0; f < 3; ++f)
        cudaMemcpyAsync(dst[f], F[f] + off[i], bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(v[i]->hist, Hp + off[i], bytes, cudaMemcpyDeviceToDevice, J->s);
      cudaMemcpyAsync(v[i]->hist + v[i]->N, Hl + off[i], bytes, cudaMemcpyDeviceToDevice, J->s);
    }
    if (cudaGetLastError() != cudaSuccess && !e) e = SGN_ERR_CUDA;
  }
  J->err = e;
  S->batch_busy = true;
  launch_job(S, J);
}

// A 2d solve, or the next chunk of a 2d or multistep run, on the request's lane.
void issue_single(sgn_server* S, Req* r) {
  Job* J = new Job();
  J->kind = JOB_SINGLE;
  J->reqs = {r};
  J->s = (r->d == 2) ? S->lane_2d : r->own;
  r->last_issue = now_s();
  sgn_status e = SGN_OK;
  wait_ready(J->s, J->reqs);
  const sgn_opts& o = r->q.opts;
  if (r->q.kind == SGN_REQ_SOLVE) {
    if ((J->info_at = take_info(S, 1)) < 0) e = SGN_ERR_NOMEM;
    J->info_n = 1;
    if (!e) {
      cudaMemsetAsync(r->u, 0, sizeof(double) * r->d * (size_t)r->N, J->s);
      e = sgn_pcg_async(S->ctx, r->lay, r->eta, r->gh, r->b, r->u, o.rtol, o.maxit, o.prec,
                        S->info_dev + J->info_at, J->s);
      cudaMemcpyAsync(S->info_host + J->info_at, S->info_dev + J->info_at, sizeof(sgn_pcg_info),
                      cudaMemcpyDeviceToHost, J->s);
    }
  } else {
    const int K = std::min(kChunk, r->remaining);
    J->K = K;
    const double dt = r->q.dt;
    switch (r->q.scheme) {
      case SGN_SCHEME_RK4: e = sgn_step_rk4(r->st, &dt, K, &o, J->s); break;
      case SGN_SCHEME_LINIMP: e = sgn_step_linimp(r->st, &dt, K, &o, J->s); break;
      default: e = sgn_step_abk(r->st, (int)r->q.scheme, &dt, K, &o, J->s); break;
    }
  }
  if (cudaGetLastError() != cudaSuccess && !e) e = SGN_ERR_CUDA;
  J->err = e;
  launch_job(S, J);
}

// A job whose event has fired (or that failed when issued): update its requests.
void complete(sgn_server* S, Job* J) {
  if (J->kind == JOB_SOLVES_1D) {
    for (size_t i = 0; i < J->reqs.size(); ++i) {
      Req* r = J->reqs[i];
      if (J->err) {
        finish(S, r, J->err);
        continue;
      }
      r->info = S->info_host[J->info_at + i];
      finish(S, r, (sgn_status)r->info.status);
    }
    if (J->lay) {
      S->reap_lays.push_back(J->lay);
      S->reap_bytes += 1 << 20;
    }
  } else if (J->kind == JOB_RUN_BATCH) {
    S->batch_busy = false;
    sgn_state_stats stt{};
    sgn_status e = J->err;
    if (!e) e = sgn_state_get_stats(S->run_st, &stt);     // the lane has finished: no wait
    for (Req* r : J->reqs) {
      r->busy = false;
      r->remaining -= J->K;
      r->iters += stt.iterations / (long long)J->reqs.size();   // shared launches: mean
      if (e || stt.status != SGN_OK) {
        finish(S, r, e ? e : (sgn_status)stt.status);
      } else if (r->remaining <= 0) {
        r->info.iters = (int)r->iters;
        finish(S, r, SGN_OK);
      }
    }
  } else {
    Req* r = J->reqs[0];
    r->busy = false;
    if (r->q.kind == SGN_REQ_SOLVE) {
      if (J->err) {
        finish(S, r, J->err);
      } else {
        r->info = S->info_host[J->info_at];
        finish(S, r, (sgn_status)r->info.status);
      }
    } else {
      sgn_state_stats stt{};
      sgn_status e = J->err;
      if (!e) e = sgn_state_get_stats(r->st, &stt);
      r->remaining -= J->K;
      if (e || stt.status != SGN_OK) {
        finish(S, r, e ? e : (sgn_status)stt.status);
      } else if (r->remaining <= 0) {
        r->info.iters = (int)stt.iterations;
        finish(S, r, SGN_OK);
      }
    }
  }
  if (J->info_at >= 0) give_info(S, J->info_at, J->info_n);
  if (J->ev) S->events.push_back(J->ev);
  delete J;
}

// Completes every job whose event has fired; returns how many.
int poll_jobs(sgn_server* S) {
  int n = 0;
  for (size_t i = 0; i < S->inflight.size();) {
    Job* J = S->inflight[i];
    const cudaError_t q = J->err ? cudaSuccess : cudaEventQuery(J->ev);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (q != cudaSuccess) {
      cudaGetLastError();
      J->err = SGN_ERR_CUDA;
    }
    S->inflight.erase(S->inflight.begin() + i);
    complete(S, J);
    ++n;
  }
  return n;
}

void worker_main(sgn_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Req*> admit_now;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop && S->pending.empty() && S->active.empty() && S->inflight.empty()) break;
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
      if (r->d == 1 && r->q.kind == SGN_REQ_RUN && !is_batched_run(r) &&
          cudaStreamCreateWithPriority(&r->own, cudaStreamNonBlocking, S->prio_lo) !=
              cudaSuccess) {
        cudaGetLastError();
        finish(S, r, SGN_ERR_CUDA);
        continue;
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.push_back(r);
    }
    const int completed = poll_jobs(S);
    std::vector<Req*> act;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.erase(std::remove_if(S->active.begin(), S->active.end(),
                                     [](Req* r) { return r->done; }),
                      S->active.end());
      act = S->active;
    }
    // issue work for every idle request
    std::vector<Req*> solves1d, runs1d, singles;
    for (Req* r : act) {
      if (r->done || r->busy) continue;
      if (r->q.kind == SGN_REQ_SOLVE && r->d == 1) solves1d.push_back(r);
      else if (is_batched_run(r)) runs1d.push_back(r);
      else singles.push_back(r);
    }
    int issued = 0;
    while (!solves1d.empty()) {
      const sgn_opts o = solves1d[0]->q.opts;
      std::vector<Req*> grp, rest;
      for (Req* r : solves1d)
        (memcmp(&r->q.opts, &o, sizeof(o)) == 0 ? grp : rest).push_back(r);
      issue_solves_1d(S, grp);
      ++issued;
      solves1d.swap(rest);
    }
    if (!S->batch_busy && !runs1d.empty()) {
      // one option set per chunk; the others wait for the batch lane
      const sgn_opts o = runs1d[0]->q.opts;
      std::vector<Req*> grp;
      for (Req* r : runs1d)
        if (memcmp(&r->q.opts, &o, sizeof(o)) == 0) grp.push_back(r);
      issue_run_batch(S, grp);
      ++issued;
    }
    // 2d work shares one lane, one job at a time, so two requests' persistent inner solves
    // never wait on each other's CTAs.  Its turn goes to a waiting 2d solve first (short),
    // else to the 2d run served longest ago.
    bool busy2d = false;
    for (Job* J : S->inflight)
      if (J->kind == JOB_SINGLE && J->reqs[0]->d == 2) busy2d = true;
    Req* next2d = nullptr;
    for (Req* r : singles) {
      if (r->d == 2) {
        const bool better = !next2d ||
                            (r->q.kind == SGN_REQ_SOLVE && next2d->q.kind != SGN_REQ_SOLVE) ||
                            (r->q.kind == next2d->q.kind && r->last_issue < next2d->last_issue);
        if (better) next2d = r;
        continue;
      }
      issue_single(S, r);
      ++issued;
    }
    if (next2d && !busy2d) {
      issue_single(S, next2d);
      ++issued;
    }
    reap(S, S->reap_bytes >= kReapBytes);
    if (!completed && !issued) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(50), [&] { return S->stop || !S->pending.empty(); });
    }
  }
  reap(S, true);
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
  bool ok = cudaMemGetInfo(&fr, &tot) == cudaSuccess &&
            cudaDeviceGetStreamPriorityRange(&S->prio_lo, &S->prio_hi) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) == cudaSuccess;
  // priorities (numerically lower is higher): 2d lane highest (its cooperative launches
  // must get every SM soon), then the 1d solve groups, then the run batch
  const int mid = S->prio_hi + 1 < S->prio_lo ? S->prio_hi + 1 : S->prio_lo;
  for (auto& l : S->lane_solve)
    ok = ok && cudaStreamCreateWithPriority(&l, cudaStreamNonBlocking, mid) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&S->lane_2d, cudaStreamNonBlocking, S->prio_hi) ==
                 cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&S->lane_batch, cudaStreamNonBlocking, S->prio_lo) ==
                 cudaSuccess;
  ok = ok && cudaMalloc(&S->info_dev, sizeof(sgn_pcg_info) * kInfoSlots) == cudaSuccess;
  ok = ok && cudaMallocHost(&S->info_host, sizeof(sgn_pcg_info) * kInfoSlots) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    for (cudaStream_t t : {S->stream, S->copy, S->lane_solve[0], S->lane_solve[1], S->lane_2d,
                           S->lane_batch})
      if (t) cudaStreamDestroy(t);
    cudaFree(S->info_dev);
    cudaFreeHost(S->info_host);
    sgn_destroy(S->ctx);
    delete S;
    return SGN_ERR_CUDA;
  }
  S->info_used.assign(kInfoSlots, 0);
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
  auto side2 = [](int n) { return pow2_in(n, 8, 1024) || sgn::mr2d_side_ok(n); };
  if (d == 1) {
    if (g.ny != 1 || !(pow2_in(g.nx, 8, 16384) || sgn::mr_size_ok(g.nx)))
      return SGN_ERR_UNSUPPORTED_SIZE;
  } else if (d == 2) {
    if (!side2(g.nx) || !side2(g.ny)) return SGN_ERR_UNSUPPORTED_SIZE;
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
    // the worker still holds the request in its deferred frees: it deletes it there
    if (!r->reaped) {
      r->released = true;
      return SGN_OK;
    }
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
  for (cudaEvent_t e : S->events) cudaEventDestroy(e);
  for (cudaStream_t t : {S->stream, S->copy, S->lane_solve[0], S->lane_solve[1], S->lane_2d,
                         S->lane_batch})
    cudaStreamDestroy(t);
  cudaFree(S->info_dev);
  cudaFreeHost(S->info_host);
  sgn_destroy(S->ctx);
  delete S;
}
