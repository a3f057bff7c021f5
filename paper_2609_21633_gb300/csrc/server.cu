// Continuous-batching Stokes solve server.
//
// Requests (shell size, viscosity contrast, buoyancy and an analytic temperature
// perturbation) are queued on submit.  max_active worker threads, each with its own CUDA
// stream, take the first queued request that can be admitted and solve it with
// tn_stokes_solve; solves of different requests therefore overlap on the device.
// Admission is by device memory: every mesh hierarchy the server holds (in use or idle)
// counts against a budget fixed at creation (memory_fraction x free memory); idle hierarchies
// are kept resident per shape and reused by later requests of the same shape, and evicted,
// least recently used first, when a new shape needs the room.  A request whose estimated
// footprint exceeds the whole budget completes at once with TN_ENOMEM.
// Every request runs on its own mesh, vectors and stream with fixed-order reductions, so its
// result does not depend on what else is running.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace tn {
namespace {

// Prescribed temperature at every node of level 0: conductive profile plus
// amp * cos(m phi) * P_l^m(cos theta) / pmax * sin(pi (r - r_in) / (r_out - r_in)).
__global__ void k_temperature(Dims D, const double* __restrict__ svec, const double* __restrict__ rad, double r_in,
                              double r_out, int l, int m, double amp_over_pmax, double* T) {
  const int M = D.N + 1;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= (int64_t)10 * D.n_r * M * M) return;
  const int j = (int)(tid % M), i = (int)((tid / M) % M), k = (int)((tid / ((int64_t)M * M)) % D.n_r),
            d = (int)(tid / ((int64_t)M * M * D.n_r));
  const int64_t so = ((int64_t)d * M + i) * D.P + j;
  const double sx = svec[so], sy = svec[so + D.n_lat_layout], sz = svec[so + 2 * D.n_lat_layout];
  const double r = rad[k];
  const double x = fmin(1.0, fmax(-1.0, sz));
  const double phi = atan2(sy, sx);
  // associated Legendre P_l^m(x), unnormalised, no Condon-Shortley phase (standard recurrence)
  double pmm = 1.0, somx2 = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x))), fact = 1.0;
  for (int q = 0; q < m; ++q) pmm *= fact * somx2, fact += 2.0;
  double plm = pmm;
  if (l > m) {
    double pmmp1 = x * (2 * m + 1) * pmm;
    plm = pmmp1;
    for (int ll = m + 2; ll <= l; ++ll) {
      const double pll = (x * (2 * ll - 1) * pmmp1 - (ll + m - 1) * pmm) / (ll - m);
      pmm = pmmp1, pmmp1 = pll, plm = pll;
    }
  }
  const double Tc = r_in * (r - r_out) / (r * (r_in - r_out));
  const double pi = 3.14159265358979323846;
  T[(int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride + (int64_t)i * D.P + j] =
      Tc + amp_over_pmax * cos(m * phi) * plm * sin(pi * (r - r_in) / (r_out - r_in));
}

double pmax_of(int l, int m) {
  double best = 0.0;
  for (int s = 0; s <= 4000; ++s) {
    const double x = -1.0 + 2.0 * s / 4000.0;
    double pmm = 1.0, somx2 = std::sqrt(std::max(0.0, (1.0 - x) * (1.0 + x))), fact = 1.0;
    for (int q = 0; q < m; ++q) pmm *= fact * somx2, fact += 2.0;
    double plm = pmm;
    if (l > m) {
      double pmmp1 = x * (2 * m + 1) * pmm;
      plm = pmmp1;
      for (int ll = m + 2; ll <= l; ++ll) {
        const double pll = (x * (2 * ll - 1) * pmmp1 - (ll + m - 1) * pmm) / (ll - m);
        pmm = pmmp1, pmmp1 = pll, plm = pll;
      }
    }
    best = std::max(best, std::fabs(plm));
  }
  return best > 0 ? best : 1.0;
}

struct Shape {
  int l, nr;
  double r_in, r_out;
  bool operator<(const Shape& o) const {
    if (l != o.l) return l < o.l;
    if (nr != o.nr) return nr < o.nr;
    if (r_in != o.r_in) return r_in < o.r_in;
    return r_out < o.r_out;
  }
};

// Device bytes a resident hierarchy may hold (tables, viscosity, multigrid and FGMRES(30)
// workspaces), estimated from the finest node layout.  Per layout entry and component: FP64
// solves hold 63 Krylov and about 30 multigrid / work vectors in FP64; mixed solves hold them in
// FP32 plus 4 FP64 work vectors.  The coarser levels add about 1/7; geometry, viscosity and
// masks about 40 bytes.
size_t footprint(const Shape& s, int mode) {
  const int N = 1 << s.l;
  const size_t P = (size_t)(N + 4) / 4 * 4;
  const size_t n0 = (size_t)10 * s.nr * (N + 1) * P;
  const double per = mode == TN_SOLVE_MIXED ? 3.0 * (93.0 * 4.0 + 4.0 * 8.0) : 3.0 * 93.0 * 8.0;
  return (size_t)((double)n0 * (per * 8.0 / 7.0 + 40.0)) + ((size_t)64 << 20);
}

struct Job {
  uint64_t ticket;
  tn_request req;
  tn_result res;
  std::vector<double> u, p;  // host copy of the solution (keep_solutions)
  bool done = false;
  std::atomic<int> cancel{0};  // set by tn_server_cancel; polled by the solver while the job runs
};

struct Pooled {
  tn_mesh* mesh;
  Shape shape;
  uint64_t last_use;
};

}  // namespace
}  // namespace tn

struct tn_server {
  tn_server_opts opts;
  int device = 0;
  size_t budget = 0, reserved = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<tn::Job*> queue;
  std::map<uint64_t, tn::Job*> jobs;
  std::vector<tn::Pooled> idle;
  uint64_t next_ticket = 1, use_clock = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::chrono::steady_clock::time_point t0;
  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace tn {
namespace {

// Under the lock: find a mesh for s (idle of the same shape, or room for a new one after evicting
// idle meshes of other shapes).  Returns 1 and sets *out (nullptr: create a new one) on success.
int acquire_locked(tn_server* S, const Shape& s, tn_mesh** out, std::vector<tn_mesh*>& to_free) {
  for (size_t q = 0; q < S->idle.size(); ++q) {
    const Shape& t = S->idle[q].shape;
    if (!(t < s) && !(s < t)) {
      *out = S->idle[q].mesh;
      S->idle.erase(S->idle.begin() + q);
      return 1;
    }
  }
  const size_t need = footprint(s, S->opts.mode);
  while (S->reserved + need > S->budget && !S->idle.empty()) {
    size_t lru = 0;
    for (size_t q = 1; q < S->idle.size(); ++q)
      if (S->idle[q].last_use < S->idle[lru].last_use) lru = q;
    S->reserved -= footprint(S->idle[lru].shape, S->opts.mode);
    to_free.push_back(S->idle[lru].mesh);
    S->idle.erase(S->idle.begin() + lru);
  }
  if (S->reserved + need > S->budget) return 0;
  S->reserved += need;
  *out = nullptr;
  return 1;
}

// One request's device state between its set-up and its bookkeeping.
struct JobRun {
  Job* J = nullptr;
  tn_mesh* mesh = nullptr;
  double *T = nullptr, *f[3] = {nullptr, nullptr, nullptr}, *u[3] = {nullptr, nullptr, nullptr}, *p = nullptr;
  tn_status s = TN_OK;
};

// Mesh (created if none is resident), vectors from the stream-ordered pool, temperature, viscosity
// and buoyancy, all enqueued on st.
void prepare_job(tn_server* S, JobRun& R, cudaStream_t st) {
  const tn_request& Q = R.J->req;
  if (!R.mesh) {
    tn_mesh_opts mo = {TN_BC_FREESLIP, TN_BC_FREESLIP, 1, 0, S->opts.eta_storage, S->opts.hg_kappa,
                       S->opts.radial_quad_points};
    R.s = tn_mesh_create(Q.lateral_level, Q.radial_layers, Q.r_in, Q.r_out, &mo, &R.mesh);
    if (R.s != TN_OK) {
      R.mesh = nullptr;
      return;
    }
  }
  const Level& L0 = R.mesh->lv[0];
  const Level& L1 = R.mesh->lv[1];
  // per-request vectors come from the stream-ordered pool (no device-wide synchronisation)
  cudaError_t e = cudaMallocAsync((void**)&R.T, sizeof(double) * L0.n_layout, st);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMallocAsync((void**)&R.f[c], sizeof(double) * L0.n_layout, st);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMallocAsync((void**)&R.u[c], sizeof(double) * L0.n_layout, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&R.p, sizeof(double) * L1.n_layout, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(R.T, 0, sizeof(double) * L0.n_layout, st);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMemsetAsync(R.f[c], 0, sizeof(double) * L0.n_layout, st);
  if (e == cudaSuccess) {
    const int64_t n = (int64_t)10 * L0.n_r * (L0.N + 1) * (L0.N + 1);
    const double amp = Q.t_amplitude / pmax_of(Q.t_degree, Q.t_order);
    k_temperature<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dims(L0), L0.s64, L0.rad64, Q.r_in, Q.r_out,
                                                                Q.t_degree, Q.t_order, amp, R.T);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    R.s = TN_ECUDA;
    return;
  }
  tn_visc_law law{Q.E, 0.0, 1.0};
  R.s = tn_set_temperature(R.mesh, R.T, &law, st);
  if (R.s == TN_OK) R.s = tn_buoyancy(R.mesh, R.T, Q.Ra, R.f, st);
}

// Solution copy (keep_solutions), vectors back to the pool, the mesh back to the idle pool (or its
// reservation released), the result published.
void finish_job(tn_server* S, JobRun& R, cudaStream_t st) {
  Job* J = R.J;
  const tn_request& Q = J->req;
  if (R.mesh && (R.s == TN_OK || R.s == TN_ENOTCONVERGED) && S->opts.keep_solutions) {
    const Level& L0 = R.mesh->lv[0];
    const Level& L1 = R.mesh->lv[1];
    J->u.resize((size_t)3 * L0.n_layout);
    J->p.resize((size_t)L1.n_layout);
    for (int c = 0; c < 3; ++c)
      cudaMemcpyAsync(J->u.data() + (size_t)c * L0.n_layout, R.u[c], sizeof(double) * L0.n_layout,
                      cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(J->p.data(), R.p, sizeof(double) * L1.n_layout, cudaMemcpyDeviceToHost, st);
  }
  for (double* q : {R.T, R.f[0], R.f[1], R.f[2], R.u[0], R.u[1], R.u[2], R.p})
    if (q) cudaFreeAsync(q, st);
  cudaStreamSynchronize(st);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    const Shape sh{Q.lateral_level, Q.radial_layers, Q.r_in, Q.r_out};
    if (R.mesh) S->idle.push_back(Pooled{R.mesh, sh, ++S->use_clock});
    else S->reserved -= footprint(sh, S->opts.mode);
    J->res.status = R.s;
    J->res.t_end = S->now();
    J->res.state = 2;
    J->done = true;
    --S->running;
  }
}

// One request, or a lockstep batch of same-shape requests (tn_stokes_solve_batch), on stream st.
void run_jobs(tn_server* S, std::vector<JobRun>& runs, cudaStream_t st) {
  for (JobRun& R : runs) prepare_job(S, R, st);
  tn_solve_opts so;
  tn_solve_default_opts(&so);
  so.mode = S->opts.mode;
  so.rtol = S->opts.rtol;
  std::vector<JobRun*> ready;
  for (JobRun& R : runs)
    if (R.s == TN_OK) ready.push_back(&R);
  for (JobRun* R : ready) R->mesh->cancel = &R->J->cancel;
  if (ready.size() == 1 || (!ready.empty() && so.mode == TN_SOLVE_MIXED)) {
    for (JobRun* R : ready) {
      tn_solve_stats ss{};
      R->s = tn_stokes_solve(R->mesh, &so, (const double* const*)R->f, nullptr, R->u, R->p, &ss, st);
      R->J->res.iterations = ss.iterations, R->J->res.refinements = ss.refinements;
      R->J->res.rel_residual = ss.rel_residual;
    }
  } else if (!ready.empty()) {
    const size_t n = ready.size();
    std::vector<tn_mesh*> ms(n);
    std::vector<const double* const*> fs(n);
    std::vector<double* const*> us(n);
    std::vector<double*> ps(n);
    std::vector<tn_solve_stats> ss(n);
    std::vector<tn_status> st_(n);
    for (size_t i = 0; i < n; ++i)
      ms[i] = ready[i]->mesh, fs[i] = ready[i]->f, us[i] = ready[i]->u, ps[i] = ready[i]->p;
    tn_stokes_solve_batch(ms.data(), (int)n, &so, fs.data(), nullptr, us.data(), ps.data(), ss.data(), st_.data(), st);
    for (size_t i = 0; i < n; ++i) {
      ready[i]->s = st_[i];
      ready[i]->J->res.iterations = ss[i].iterations, ready[i]->J->res.refinements = ss[i].refinements;
      ready[i]->J->res.rel_residual = ss[i].rel_residual;
      ready[i]->J->res.batch = (int)n;
    }
  }
  for (JobRun* R : ready) R->mesh->cancel = nullptr;
  for (JobRun& R : runs) finish_job(S, R, st);
  S->cv_done.notify_all();
  S->cv_work.notify_all();
}

void worker(tn_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  while (true) {
    std::vector<JobRun> runs;
    std::vector<tn_mesh*> to_free;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stop && S->queue.empty()) break;
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
          const tn_request& R = (*it)->req;
          tn_mesh* mesh = nullptr;
          if (acquire_locked(S, Shape{R.lateral_level, R.radial_layers, R.r_in, R.r_out}, &mesh, to_free)) {
            runs.push_back(JobRun{*it, mesh});
            S->queue.erase(it);
            break;
          }
        }
        if (!runs.empty()) break;
        S->cv_work.wait(lk);
      }
      if (runs.empty()) break;
      // lockstep batch: further queued requests of the same shape, as long as they fit the budget
      const tn_request& R0 = runs[0].J->req;
      const Shape s0{R0.lateral_level, R0.radial_layers, R0.r_in, R0.r_out};
      for (auto it = S->queue.begin(); it != S->queue.end() && (int)runs.size() < S->opts.max_batch;) {
        const tn_request& R = (*it)->req;
        const Shape sh{R.lateral_level, R.radial_layers, R.r_in, R.r_out};
        tn_mesh* mesh = nullptr;
        if (!(sh < s0) && !(s0 < sh) && acquire_locked(S, sh, &mesh, to_free)) {
          runs.push_back(JobRun{*it, mesh});
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
      for (JobRun& r : runs) {
        ++S->running;
        r.J->res.state = 1;
        r.J->res.t_start = S->now();
      }
    }
    for (tn_mesh* m : to_free) tn_mesh_destroy(m);
    run_jobs(S, runs, st);
  }
  cudaStreamDestroy(st);
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_server_default_opts(tn_server_opts* o) {
  if (!o) return TN_EINVAL;
  o->max_active = 4;
  o->memory_fraction = 0.8;
  o->mode = TN_SOLVE_MIXED;
  o->rtol = 1e-8;
  o->keep_solutions = 0;
  o->eta_storage = TN_ETA_F32;
  o->hg_kappa = 0.0;
  o->radial_quad_points = 1;
  o->max_batch = 1;
  return TN_OK;
}

tn_status tn_server_create(const tn_server_opts* opts, tn_server** out) {
  if (!out) return TN_EINVAL;
  tn_server_opts o;
  tn_server_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_active < 1 || o.max_active > 64 || !(o.memory_fraction > 0.0) || o.memory_fraction > 1.0 ||
      !(o.rtol > 0.0) || o.eta_storage < TN_ETA_F32 || o.eta_storage > TN_ETA_F16 || !(o.hg_kappa >= 0.0) ||
      o.radial_quad_points < 0 || o.radial_quad_points > 2 || (o.radial_quad_points == 2 && o.hg_kappa > 0.0) ||
      o.max_batch < 1 || o.max_batch > 64) {
    set_error("tn_server_create: invalid options");
    return TN_EINVAL;
  }
  tn_server* S = new tn_server();
  S->opts = o;
  cudaGetDevice(&S->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete S;
    set_error("tn_server_create: cudaMemGetInfo failed");
    return TN_ECUDA;
  }
  S->budget = (size_t)(o.memory_fraction * (double)free_b);
  S->t0 = std::chrono::steady_clock::now();
  for (int w = 0; w < o.max_active; ++w) S->workers.emplace_back(worker, S);
  *out = S;
  return TN_OK;
}

tn_status tn_server_submit(tn_server* S, const tn_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket) return TN_EINVAL;
  if (req->lateral_level < 1 || req->radial_layers < 3 || (req->radial_layers - 1) % 2 != 0 ||
      !(req->r_in > 0) || !(req->r_out > req->r_in) || !std::isfinite(req->r_out) || req->t_degree < 0 ||
      req->t_order < 0 || req->t_order > req->t_degree || !std::isfinite(req->E) || !std::isfinite(req->Ra) ||
      !std::isfinite(req->t_amplitude)) {
    set_error("tn_server_submit: invalid request");
    return TN_EINVAL;
  }
  Job* J = new Job();
  J->req = *req;
  std::memset(&J->res, 0, sizeof(J->res));
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete J;
      set_error("tn_server_submit: server is shutting down");
      return TN_ESTATE;
    }
    J->ticket = S->next_ticket++;
    J->res.t_submit = S->now();
    J->res.state = 0;
    S->jobs[J->ticket] = J;
    const Shape s{req->lateral_level, req->radial_layers, req->r_in, req->r_out};
    if (footprint(s, S->opts.mode) > S->budget) {  // can never be admitted
      J->res.status = TN_ENOMEM;
      J->res.state = 2;
      J->res.t_start = J->res.t_end = J->res.t_submit;
      J->done = true;
    } else {
      S->queue.push_back(J);
    }
    *ticket = J->ticket;
  }
  S->cv_work.notify_all();
  return TN_OK;
}

tn_status tn_server_poll(tn_server* S, uint64_t ticket, tn_result* res) {
  if (!S || !res) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    set_error("tn_server_poll: unknown ticket");
    return TN_EINVAL;
  }
  *res = it->second->res;
  return it->second->done ? TN_OK : TN_EBUSY;
}

tn_status tn_server_wait(tn_server* S, uint64_t ticket, tn_result* res) {
  if (!S || !res) return TN_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    set_error("tn_server_wait: unknown ticket");
    return TN_EINVAL;
  }
  Job* J = it->second;
  S->cv_done.wait(lk, [&] { return J->done; });
  *res = J->res;
  return TN_OK;
}

tn_status tn_server_solution(tn_server* S, uint64_t ticket, double* u_host, double* p_host) {
  if (!S || !u_host || !p_host) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end() || !it->second->done || it->second->u.empty()) {
    set_error("tn_server_solution: no stored solution for this ticket (unknown, pending, or keep_solutions = 0)");
    return TN_EINVAL;
  }
  std::memcpy(u_host, it->second->u.data(), sizeof(double) * it->second->u.size());
  std::memcpy(p_host, it->second->p.data(), sizeof(double) * it->second->p.size());
  return TN_OK;
}

tn_status tn_server_stats(tn_server* S, int* queued, int* running, int* resident, double* reserved_bytes) {
  if (!S) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (queued) *queued = (int)S->queue.size();
  if (running) *running = S->running;
  if (resident) *resident = (int)S->idle.size() + S->running;
  if (reserved_bytes) *reserved_bytes = (double)S->reserved;
  return TN_OK;
}

tn_status tn_server_cancel(tn_server* S, uint64_t ticket) {
  if (!S) return TN_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    set_error("tn_server_cancel: unknown ticket");
    return TN_EINVAL;
  }
  Job* J = it->second;
  if (J->done) return TN_OK;
  J->cancel.store(1);
  for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
    if (*q == J) {  // still queued: it never runs
      S->queue.erase(q);
      J->res.status = TN_ECANCELED;
      J->res.state = 2;
      J->res.t_start = J->res.t_end = S->now();
      J->done = true;
      S->cv_done.notify_all();
      break;
    }
  return TN_OK;
}

tn_status tn_server_destroy(tn_server* S) {
  if (!S) return TN_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& q : S->idle) tn_mesh_destroy(q.mesh);
  for (auto& kv : S->jobs) delete kv.second;
  delete S;
  return TN_OK;
}

}  // extern "C"
