// Energy equation (Eq. energy) and the coupled Stokes-energy time loop.
//
// Space: the one-point wedge residual R = (K + C(u) + S(u)) T of the tile kernel (OpEnergy in
// kernels.cu) and the lumped mass m_j = sum_e V_e / 6.  Time: Heun's method (explicit trapezoid),
//   T* = T - dt M^-1 R(T),  T_new = (T + T* - dt M^-1 R(T*)) / 2,
// on the interior node layers; the two surface layers keep their values (prescribed temperatures).
// The substep is bounded by the diffusion eigenvalue (power iteration on M^-1 K) and the coupled step
// by an advective CFL condition.  Reductions sum per-block partials in a fixed order (deterministic).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace tn {
namespace {

constexpr int RB = 304;  // blocks of a reduction (fixed: the summation order never changes)
constexpr int RT = 256;

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

__device__ __forceinline__ int layer_of(int64_t idx, const Dims& D) { return (int)((idx / D.layer_stride) % D.n_r); }

// stage 1: out = T - dt R / m; stage 2: out = (T + T1 - dt R / m) / 2; surface layers and padding
// (m = 0) copy T
__global__ void k_heun(int stage, Dims D, int64_t n, const double* __restrict__ T, const double* __restrict__ T1,
                       const double* __restrict__ R, const double* __restrict__ m, double dt, double* out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = layer_of(idx, D);
  const double mm = m[idx];
  if (k == 0 || k == D.n_r - 1 || !(mm > 0.0)) {
    out[idx] = T[idx];
    return;
  }
  const double step = dt * R[idx] / mm;
  out[idx] = stage == 1 ? T[idx] - step : 0.5 * ((T[idx] + T1[idx]) - step);
}

// out = scale M^-1 R on the interior layers, 0 on the surface layers and padding
__global__ void k_minv(Dims D, int64_t n, const double* __restrict__ R, const double* __restrict__ m, double scale,
                       double* out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = layer_of(idx, D);
  out[idx] = (k == 0 || k == D.n_r - 1 || !(m[idx] > 0.0)) ? 0.0 : scale * R[idx] / m[idx];
}

// conductive profile T_c(r_k) = r_in (r_k - r_out) / (r_k (r_in - r_out)) at every node (padding 0)
__global__ void k_conductive(Dims D, int64_t n, const double* __restrict__ radii, double r_in, double r_out,
                             const double* __restrict__ m, double* out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const double r = radii[layer_of(idx, D)];
  out[idx] = m[idx] > 0.0 ? r_in * (r - r_out) / (r * (r_in - r_out)) : 0.0;
}

// deterministic partial reductions over canonical nodes (wmask); layer < 0: every layer
//   mode 0: sum a0;  mode 1: sum m (a0^2 + a1^2 + a2^2) and sum m;  mode 2: max |(a0, a1, a2)|;
//   mode 3: sum a0^2
__global__ void __launch_bounds__(RT) k_reduce(int mode, Dims D, int64_t n, int layer, const uint8_t* __restrict__ mask,
                                               const double* __restrict__ a0, const double* __restrict__ a1,
                                               const double* __restrict__ a2, const double* __restrict__ m,
                                               double* part) {
  __shared__ double sh[2][RT];
  double x = 0, y = 0;
  for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    if (!mask[i] || (layer >= 0 && layer_of(i, D) != layer)) continue;
    if (mode == 0) {
      x += a0[i];
    } else if (mode == 1) {
      x += m[i] * ((a0[i] * a0[i] + a1[i] * a1[i]) + a2[i] * a2[i]);
      y += m[i];
    } else if (mode == 2) {
      x = fmax(x, sqrt((a0[i] * a0[i] + a1[i] * a1[i]) + a2[i] * a2[i]));
    } else {
      x += a0[i] * a0[i];
    }
  }
  sh[0][threadIdx.x] = x, sh[1][threadIdx.x] = y;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      if (mode == 2) sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + s]);
      else sh[0][threadIdx.x] += sh[0][threadIdx.x + s], sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0][0], part[RB + blockIdx.x] = sh[1][0];
}

// Power iteration start vector: SplitMix64 (Steele, Lea, Flood 2014) of the node's lateral
// coordinates and layer, mapped to [-1, 1), so that every copy of a diamond-edge node gets the same
// value (the copies' coordinates are bitwise equal); 0 on the surface layers and padding.
__global__ void k_start(Dims D, int64_t n, const double* __restrict__ svec, const double* __restrict__ m, double* v) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int k = layer_of(idx, D);
  if (k == 0 || k == D.n_r - 1 || !(m[idx] > 0.0)) {
    v[idx] = 0.0;
    return;
  }
  const int64_t d = idx / D.diamond_stride;
  const int64_t lat = d * (D.layer_stride) + idx % D.layer_stride;  // lateral layout ((d (N+1) + i) P + j)
  uint64_t z = (uint64_t)k * 0x9e3779b97f4a7c15ull;
  for (int c = 0; c < 3; ++c) {
    z ^= (uint64_t)__double_as_longlong(svec[lat + c * D.n_lat_layout]) + 0x9e3779b97f4a7c15ull + (z << 6) + (z >> 2);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
  }
  v[idx] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

struct Red {
  double* part = nullptr;  // device, 2 RB
  std::vector<double> h = std::vector<double>(2 * RB);
};

cudaError_t reduce(Red& red, int mode, const Level& L, int layer, const double* a0, const double* a1, const double* a2,
                   const double* m, double* x, double* y, cudaStream_t st) {
  k_reduce<<<RB, RT, 0, st>>>(mode, dims(L), L.n_layout, layer, L.wmask, a0, a1 ? a1 : a0, a2 ? a2 : a0, m ? m : a0,
                              red.part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(red.h.data(), red.part, sizeof(double) * 2 * RB, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  double sx = 0, sy = 0;
  for (int b = 0; b < RB; ++b) {
    if (mode == 2) sx = std::max(sx, red.h[b]);
    else sx += red.h[b], sy += red.h[RB + b];
  }
  *x = sx;
  if (y) *y = sy;
  return cudaSuccess;
}

// Mesh-owned energy workspace on level 0: lumped mass, three work vectors, the reduction buffer,
// and the diffusion eigenvalue estimate (0: not yet computed).
cudaError_t ensure_energy(tn_mesh* mesh, cudaStream_t st) {
  EnergyState& S = mesh->en;
  const Level& L = mesh->lv[0];
  if (S.mass) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&S.mass, sizeof(double) * L.n_layout);
  for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaMalloc((void**)&S.w[q], sizeof(double) * L.n_layout);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S.part, sizeof(double) * 2 * RB);
  for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaMemsetAsync(S.w[q], 0, sizeof(double) * L.n_layout, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.mass, 0, sizeof(double) * L.n_layout, st);
  if (e == cudaSuccess) e = launch_lumped_mass(L, S.mass, st);
  if (e != cudaSuccess) {
    energy_free(mesh);
    return e;
  }
  return cudaSuccess;
}

// largest eigenvalue of M^-1 K on the interior layers: power iteration, 30 steps, the iterate
// normalised every step (w = M^-1 K v / |v|, so |w| is the estimate and the values stay near lambda)
cudaError_t diffusion_lambda(tn_mesh* mesh, cudaStream_t st, double* lam) {
  EnergyState& S = mesh->en;
  if (S.lambda > 0) {
    *lam = S.lambda;
    return cudaSuccess;
  }
  const Level& L = mesh->lv[0];
  const Dims D = dims(L);
  Red red;
  red.part = S.part;
  double* v = S.w[0];
  double* w = S.w[1];
  k_start<<<nb(L.n_layout), 256, 0, st>>>(D, L.n_layout, L.s64, S.mass, v);
  cudaError_t e = cudaGetLastError();
  double nv = 0, est = 0;
  if (e == cudaSuccess) e = reduce(red, 3, L, -1, v, nullptr, nullptr, nullptr, &nv, nullptr, st);
  for (int it = 0; it < 30 && e == cudaSuccess; ++it) {
    if (!(nv > 0) || !std::isfinite(nv)) break;
    e = launch_energy_residual(L, nullptr, v, w, 0, st);
    if (e == cudaSuccess) {
      k_minv<<<nb(L.n_layout), 256, 0, st>>>(D, L.n_layout, w, S.mass, 1.0 / std::sqrt(nv), w);
      e = cudaGetLastError();
    }
    double nw = 0;
    if (e == cudaSuccess) e = reduce(red, 3, L, -1, w, nullptr, nullptr, nullptr, &nw, nullptr, st);
    if (e != cudaSuccess || !(nw > 0) || !std::isfinite(nw)) break;
    est = std::sqrt(nw);
    std::swap(v, w);
    nv = nw;
  }
  if (e != cudaSuccess) return e;
  if (!(est > 0) || !std::isfinite(est)) return cudaErrorUnknown;  // no usable estimate: refuse to step
  S.lambda = est;
  *lam = S.lambda;
  return cudaSuccess;
}

cudaError_t heun_steps(tn_mesh* mesh, double* T, const double* const* u, double dt, int n, int supg,
                       cudaStream_t st) {
  const Level& L = mesh->lv[0];
  const Dims D = dims(L);
  EnergyState& S = mesh->en;
  double *R = S.w[0], *T1 = S.w[1], *R1 = S.w[2];
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < n && e == cudaSuccess; ++s) {
    e = launch_energy_residual(L, u, T, R, supg, st);
    if (e != cudaSuccess) break;
    k_heun<<<nb(L.n_layout), 256, 0, st>>>(1, D, L.n_layout, T, nullptr, R, S.mass, dt, T1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_energy_residual(L, u, T1, R1, supg, st);
    if (e != cudaSuccess) break;
    k_heun<<<nb(L.n_layout), 256, 0, st>>>(2, D, L.n_layout, T, T1, R1, S.mass, dt, T);
    e = cudaGetLastError();
  }
  return e;
}

// Nu_top: consistent diffusive flux (K T summed over the outer surface's canonical nodes) relative
// to that of the conductive profile; V_rms = sqrt(sum m |u|^2 / sum m) over canonical nodes.
cudaError_t diagnostics(tn_mesh* mesh, const double* T, const double* const* u, double* nu, double* vrms,
                        cudaStream_t st) {
  const Level& L = mesh->lv[0];
  EnergyState& S = mesh->en;
  Red red;
  red.part = S.part;
  cudaError_t e = cudaSuccess;
  if (nu) {
    double ft = 0, fc = 0;
    e = launch_energy_residual(L, nullptr, T, S.w[0], 0, st);
    if (e == cudaSuccess) e = reduce(red, 0, L, L.n_r - 1, S.w[0], nullptr, nullptr, nullptr, &ft, nullptr, st);
    if (e == cudaSuccess) {
      k_conductive<<<nb(L.n_layout), 256, 0, st>>>(dims(L), L.n_layout, L.rad64, mesh->r_in, mesh->r_out, S.mass,
                                                   S.w[3]);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_energy_residual(L, nullptr, S.w[3], S.w[1], 0, st);
    if (e == cudaSuccess) e = reduce(red, 0, L, L.n_r - 1, S.w[1], nullptr, nullptr, nullptr, &fc, nullptr, st);
    if (e == cudaSuccess) *nu = ft / fc;
  }
  if (vrms && e == cudaSuccess) {
    double a = 0, b = 0;
    e = reduce(red, 1, L, -1, u[0], u[1], u[2], S.mass, &a, &b, st);
    if (e == cudaSuccess) *vrms = std::sqrt(a / b);
  }
  return e;
}

// smallest node spacing: radial cells and lateral lattice edges at r_in
double min_spacing(const tn_mesh* mesh) {
  const Level& L = mesh->lv[0];
  double h = 1e300;
  for (int k = 0; k + 1 < L.n_r; ++k) h = std::min(h, L.radii[k + 1] - L.radii[k]);
  const int M = L.N + 1;
  auto dist2 = [&](int d, int i0, int j0, int i1, int j1) {
    double s = 0;
    for (int x = 0; x < 3; ++x) {
      const double t = L.lat_xyz[(((size_t)d * M + i1) * M + j1) * 3 + x] - L.lat_xyz[(((size_t)d * M + i0) * M + j0) * 3 + x];
      s += t * t;
    }
    return s;
  };
  double e2 = 1e300;
  for (int d = 0; d < 10; ++d)
    for (int i = 0; i < L.N; ++i)
      for (int j = 0; j < L.N; ++j)  // the cell's edges in i, in j, and its diagonal (i+1, j)-(i, j+1)
        e2 = std::min({e2, dist2(d, i, j, i + 1, j), dist2(d, i, j, i, j + 1), dist2(d, i + 1, j, i, j + 1)});
  return std::min(h, std::sqrt(e2) * mesh->r_in);
}

}  // namespace

void energy_free(tn_mesh* mesh) {
  EnergyState& S = mesh->en;
  for (void* p : {(void*)S.mass, (void*)S.w[0], (void*)S.w[1], (void*)S.w[2], (void*)S.w[3], (void*)S.part})
    if (p) cudaFree(p);
  S = EnergyState();
}

}  // namespace tn

using namespace tn;

namespace {
tn_status efail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
}
}  // namespace

extern "C" {

tn_status tn_energy_residual(tn_mesh* mesh, const double* T_dev, const double* const* u_dev, int supg, double* R_dev,
                             void* stream) {
  if (!mesh || !T_dev || !R_dev || T_dev == R_dev) {
    set_error("tn_energy_residual: NULL or aliasing argument");
    return TN_EINVAL;
  }
  if (u_dev && (!u_dev[0] || !u_dev[1] || !u_dev[2])) {
    set_error("tn_energy_residual: NULL velocity component");
    return TN_EINVAL;
  }
  cudaError_t e = launch_energy_residual(mesh->lv[0], u_dev, T_dev, R_dev, supg ? 1 : 0, (cudaStream_t)stream);
  return e == cudaSuccess ? TN_OK : efail(e, "tn_energy_residual");
}

tn_status tn_energy_steps(tn_mesh* mesh, double* T_dev, const double* const* u_dev, double dt, int n_steps, int supg,
                          void* stream) {
  if (!mesh || !T_dev || n_steps < 0 || !(dt >= 0.0) || !std::isfinite(dt)) {
    set_error("tn_energy_steps: bad arguments");
    return TN_EINVAL;
  }
  if (u_dev && (!u_dev[0] || !u_dev[1] || !u_dev[2])) {
    set_error("tn_energy_steps: NULL velocity component");
    return TN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = ensure_energy(mesh, st);
  if (e == cudaSuccess) e = heun_steps(mesh, T_dev, u_dev, dt, n_steps, supg ? 1 : 0, st);
  return e == cudaSuccess ? TN_OK : efail(e, "tn_energy_steps");
}

tn_status tn_energy_diagnostics(tn_mesh* mesh, const double* T_dev, const double* const* u_dev, double* nu_top,
                                double* v_rms, void* stream) {
  if (!mesh || (!T_dev && nu_top) || (v_rms && (!u_dev || !u_dev[0] || !u_dev[1] || !u_dev[2]))) {
    set_error("tn_energy_diagnostics: NULL argument");
    return TN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = ensure_energy(mesh, st);
  if (e == cudaSuccess) e = diagnostics(mesh, T_dev, u_dev, nu_top, v_rms, st);
  return e == cudaSuccess ? TN_OK : efail(e, "tn_energy_diagnostics");
}

tn_status tn_energy_stable_dt(tn_mesh* mesh, double* dt, void* stream) {
  if (!mesh || !dt) return TN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double lam = 0;
  cudaError_t e = ensure_energy(mesh, st);
  if (e == cudaSuccess) e = diffusion_lambda(mesh, st, &lam);
  if (e != cudaSuccess) return efail(e, "tn_energy_stable_dt");
  *dt = 1.5 / (1.1 * lam);
  return TN_OK;
}

tn_status tn_convection_default_opts(tn_convection_opts* o) {
  if (!o) return TN_EINVAL;
  o->Ra = 1e5;
  o->E = std::log(100.0);
  o->cfl = 0.5;
  o->supg = 1;
  o->mode = TN_SOLVE_MIXED;
  o->rtol = 1e-8;
  o->dt = 0.0;
  o->substeps = 0;
  return TN_OK;
}

tn_status tn_convection_steps(tn_mesh* mesh, double* T_dev, double* const* u_dev, double* p_dev, int n_steps,
                              const tn_convection_opts* opts, tn_convection_step_stats* stats, void* stream) {
  if (!mesh || !T_dev || !u_dev || !u_dev[0] || !u_dev[1] || !u_dev[2] || !p_dev || n_steps < 0) {
    set_error("tn_convection_steps: bad arguments");
    return TN_EINVAL;
  }
  tn_convection_opts o;
  tn_convection_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.cfl > 0) || !(o.rtol > 0) || !std::isfinite(o.Ra) || !std::isfinite(o.E) || o.dt < 0 || o.substeps < 0) {
    set_error("tn_convection_steps: invalid options");
    return TN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const Level& L = mesh->lv[0];
  cudaError_t e = ensure_energy(mesh, st);
  double* f[3] = {nullptr, nullptr, nullptr};
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMalloc((void**)&f[c], sizeof(double) * L.n_layout);
  for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMemsetAsync(f[c], 0, sizeof(double) * L.n_layout, st);
  double lam = 0;
  if (e == cudaSuccess && o.substeps == 0) e = diffusion_lambda(mesh, st, &lam);
  const double h = min_spacing(mesh);
  tn_status status = TN_OK;
  double time = 0;
  Red red;
  red.part = mesh->en.part;
  for (int s = 0; s < n_steps && e == cudaSuccess && status == TN_OK; ++s) {
    const auto t0 = std::chrono::steady_clock::now();
    tn_visc_law law{o.E, 0.0, 1.0};
    status = tn_set_temperature(mesh, T_dev, &law, stream);
    if (status == TN_OK) status = tn_buoyancy(mesh, T_dev, o.Ra, f, stream);
    tn_solve_opts so;
    tn_solve_default_opts(&so);
    so.mode = o.mode;
    so.rtol = o.rtol;
    tn_solve_stats ss{};
    if (status == TN_OK) status = tn_stokes_solve(mesh, &so, (const double* const*)f, nullptr, u_dev, p_dev, &ss, stream);
    if (status != TN_OK) break;
    const auto t1 = std::chrono::steady_clock::now();
    double umax = 0, nu = 0, vr = 0;
    e = reduce(red, 2, L, -1, u_dev[0], u_dev[1], u_dev[2], nullptr, &umax, nullptr, st);
    if (e == cudaSuccess) e = diagnostics(mesh, T_dev, (const double* const*)u_dev, &nu, &vr, st);
    if (e != cudaSuccess) break;
    double dt = o.dt > 0 ? o.dt : (umax > 0 ? o.cfl * h / umax : 1.5 / (1.1 * lam));
    int nsub = o.substeps > 0 ? o.substeps : std::max(1, (int)std::ceil(dt * 1.1 * lam / 1.5));
    e = heun_steps(mesh, T_dev, (const double* const*)u_dev, dt / nsub, nsub, o.supg ? 1 : 0, st);
    double tmax = 0;
    if (e == cudaSuccess) e = reduce(red, 2, L, -1, T_dev, T_dev, T_dev, nullptr, &tmax, nullptr, st);
    if (e != cudaSuccess) break;
    if (!std::isfinite(tmax)) {
      set_error("tn_convection_steps: the temperature is no longer finite after step " + std::to_string(s));
      status = TN_ENOTCONVERGED;
      break;
    }
    const auto t2 = std::chrono::steady_clock::now();
    time += dt;
    if (stats) {
      tn_convection_step_stats& q = stats[s];
      q.time = time;
      q.dt = dt;
      q.substeps = nsub;
      q.stokes_iterations = ss.iterations;
      q.rel_residual = ss.rel_residual;
      q.nu_top = nu;
      q.v_rms = vr;
      q.u_max = umax;
      q.stokes_seconds = std::chrono::duration<double>(t1 - t0).count();
      q.energy_seconds = std::chrono::duration<double>(t2 - t1).count();
    }
  }
  for (double* q : f)
    if (q) cudaFree(q);
  if (e != cudaSuccess) return efail(e, "tn_convection_steps");
  return status;
}

}  // extern "C"
