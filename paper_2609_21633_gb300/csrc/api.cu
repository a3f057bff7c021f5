// C ABI of the wedge Stokes library: argument checks, mesh hierarchy lifetime, dispatch.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "dfloat.cuh"
#include "internal.h"

namespace tn {

namespace {
thread_local std::string g_err = "no error";
}

void set_error(const std::string& msg) { g_err = msg; }

namespace {

tn_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return TN_ECUDA;
}

tn_status inval(const std::string& msg) {
  set_error(msg);
  return TN_EINVAL;
}

template <typename T>
cudaError_t upload(T*& dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)&dst, sizeof(T) * (src.empty() ? 1 : src.size()));
  if (e != cudaSuccess) return e;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

// a table as double-float pairs (hi, lo), split exactly as the kernels split binary64 values
std::vector<float> to_df(const std::vector<double>& v) {
  std::vector<float> out(2 * v.size());
  for (size_t q = 0; q < v.size(); ++q) {
    const dfl x = split(v[q]);
    out[2 * q] = x.hi, out[2 * q + 1] = x.lo;
  }
  return out;
}

template <typename T>
std::vector<float> to_f32(const std::vector<T>& v) {
  std::vector<float> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = (float)v[i];
  return out;
}

void free_level(Level& L) {
  void* ptrs[] = {L.geo64, L.geo32, L.lay64, L.lay32, L.laydf, L.s64,   L.s32,   L.grp_ptr, L.grp_off, L.grp_s64,
                  L.grp_s32, L.owned, L.eta64, L.eta32, L.eta16, L.eta_cs, L.scr64, L.scr32, L.wmask, L.rad64,
                  L.rad32, L.dcoef64, L.dcoef32, L.dcoefdf, L.dcoefdf2, L.ring64, L.grp_dij, L.bw64, L.rhat64, L.rhat32, L.rhatdf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  L = Level();
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

bool level_ok(const tn_mesh* m, int level) { return m && level >= 0 && level < (int)m->lv.size(); }

BC bc_of(const tn_mesh* m) { return BC{m->bc_in, m->bc_out}; }

template <typename T>
cudaError_t apply_B_t(tn_mesh* m, int level, const void* const* u, void* q, cudaStream_t st) {
  const Level& F = m->lv[level];
  const Level& C = m->lv[level + 1];
  T* scr = sizeof(T) == 8 ? (T*)F.scr64 : (T*)F.scr32;
  cudaError_t e = launch_div_fine<T>(F, bc_of(m), (const T* const*)u, scr, st);
  if (e != cudaSuccess) return e;
  const T* fin[1] = {scr};
  T* cout[1] = {(T*)q};
  return launch_restrict<T>(F, C, bc_of(m), 1, 0, fin, cout, st);
}

template <typename T>
cudaError_t apply_BT_t(tn_mesh* m, int level, const void* p, void* const* y, cudaStream_t st) {
  const Level& F = m->lv[level];
  const Level& C = m->lv[level + 1];
  T* scr = sizeof(T) == 8 ? (T*)F.scr64 : (T*)F.scr32;
  const T* cin[1] = {(const T*)p};
  T* fout[1] = {scr};
  cudaError_t e = launch_prolong<T>(F, C, bc_of(m), 1, 0, cin, fout, st);
  if (e != cudaSuccess) return e;
  return launch_grad_fine<T>(F, bc_of(m), scr, (T* const*)y, st);
}


}  // namespace

// Host tables and device arrays of one level (lateral level l, nr node layers).
// The diag(A) factor table of the level (see Level::dcoef64) from the FP64 geometry table.
std::vector<double> diag_factors(const std::vector<double>& geo, int64_t n_tri, int div_term) {
  std::vector<double> v((size_t)kDiagCoef * n_tri, 0.0);
  const double c = div_term ? 1.0 / 3.0 : 1.0;
  for (int64_t t = 0; t < n_tri; ++t) {
    double m[3][3], l[3][3];
    for (int k = 0; k < 3; ++k)
      for (int x = 0; x < 3; ++x) m[k][x] = geo[(size_t)(3 * k + x) * n_tri + t];
    for (int x = 0; x < 3; ++x) l[0][x] = -(m[0][x] + m[1][x]), l[1][x] = m[0][x], l[2][x] = m[1][x];
    auto put = [&](int q, double val) { v[(size_t)q * n_tri + t] = val; };
    const double m22 = m[2][0] * m[2][0] + m[2][1] * m[2][1] + m[2][2] * m[2][2];
    for (int a = 0; a < 3; ++a) {
      const double ll = l[a][0] * l[a][0] + l[a][1] * l[a][1] + l[a][2] * l[a][2];
      const double lm = l[a][0] * m[2][0] + l[a][1] * m[2][1] + l[a][2] * m[2][2];
      for (int d = 0; d < 3; ++d) {
        put(3 * a + d, ll + c * l[a][d] * l[a][d]);
        put(9 + 3 * a + d, lm + c * l[a][d] * m[2][d]);
      }
    }
    for (int d = 0; d < 3; ++d) put(18 + d, m22 + c * m[2][d] * m[2][d]);
    double L = 0;
    for (int x = 0; x < 3; ++x) {
      const double s01 = m[0][x] + m[1][x];
      L += s01 * s01 + m[0][x] * m[0][x] + m[1][x] * m[1][x];
    }
    put(21, 2.0 * L);
    put(22, 6.0 * m22);
  }
  return v;
}

tn_status create_level(Level& L, int l, int nr, double r_in, double r_out, int eta_storage, int div_term) {
  std::vector<double> geo, lay, s, grp_s;
  std::vector<int> gptr;
  std::vector<int64_t> goff;
  std::vector<uint8_t> owned;
  std::string err;
  build_level_host(L, l, nr, r_in, r_out, geo, lay, s, gptr, goff, grp_s, owned, err);
  if (!err.empty()) return inval("tn_mesh_create: " + err);
  L.h_grp_ptr = gptr;
  L.h_grp_off = goff;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(upload(L.geo64, geo));
  chk(upload(L.geo32, to_f32(geo)));
  {
    const std::vector<double> dc = diag_factors(geo, L.n_tri, div_term);
    chk(upload(L.dcoef64, dc));
    chk(upload(L.dcoef32, to_f32(dc)));
    const std::vector<float> dcf = to_df(dc);
    chk(upload(L.dcoefdf, dcf));
    {
      const int64_t nt = L.n_tri, np = nt / 2;
      std::vector<float4> d2((size_t)kDiagCoef * np);
      for (int q = 0; q < kDiagCoef; ++q)
        for (int64_t pp = 0; pp < np; ++pp) {
          const size_t a = 2 * (size_t)(q * nt + 2 * pp), b = a + 2;
          d2[(size_t)q * np + pp] = make_float4(dcf[a], dcf[b], dcf[a + 1], dcf[b + 1]);
        }
      chk(upload(L.dcoefdf2, d2));
    }
    L.dcoef_div = div_term;
  }
  chk(upload(L.lay64, lay));
  chk(upload(L.lay32, to_f32(lay)));
  chk(upload(L.laydf, to_df(lay)));
  L.h_lay = lay;
  {
    // r_hat(q_c) = sbar / |sbar| of every lateral triangle t = ((d N + i) N + j) 2 + w
    const int N = L.N, M = N + 1;
    std::vector<double> rh((size_t)3 * L.n_tri);
    for (int d = 0; d < 10; ++d)
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
          for (int w = 0; w < 2; ++w) {
            const int ci[3] = {w ? i + 1 : i, w ? i : i + 1, w ? i + 1 : i};
            const int cj[3] = {w ? j + 1 : j, w ? j + 1 : j, w ? j : j + 1};
            double sb[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a)
              for (int x = 0; x < 3; ++x) sb[x] += L.lat_xyz[(((size_t)d * M + ci[a]) * M + cj[a]) * 3 + x];
            const double nrm = std::sqrt(sb[0] * sb[0] + sb[1] * sb[1] + sb[2] * sb[2]);
            const int64_t t = (((int64_t)d * N + i) * N + j) * 2 + w;
            for (int x = 0; x < 3; ++x) rh[(size_t)x * L.n_tri + t] = sb[x] / nrm;
          }
    chk(upload(L.rhat64, rh));
    chk(upload(L.rhat32, to_f32(rh)));
    chk(upload(L.rhatdf, to_df(rh)));
  }
  chk(upload(L.s64, s));
  chk(upload(L.s32, to_f32(s)));
  chk(upload(L.grp_ptr, gptr));
  chk(upload(L.grp_off, goff));
  chk(upload(L.grp_s64, grp_s));
  chk(upload(L.grp_s32, to_f32(grp_s)));
  chk(upload(L.owned, owned));
  chk(cudaMalloc((void**)&L.eta64, sizeof(double) * L.n_wedges));
  // 16-bit viscosity only where the tile kernel runs with full 16 x 16 tiles
  L.eta_kind = (eta_storage != TN_ETA_F32 && L.N >= 16) ? eta_storage : TN_ETA_F32;
  if (L.eta_kind == TN_ETA_F32) {
    chk(cudaMalloc((void**)&L.eta32, sizeof(float) * L.n_wedges));
  } else {
    chk(cudaMalloc((void**)&L.eta16, sizeof(uint16_t) * L.n_wedges));
    chk(cudaMalloc((void**)&L.eta_cs, sizeof(float) * L.n_tri));
  }
  {
    const int64_t nring = ring_buffer_entries(L.N, L.n_r);
    if (nring > 0) {
      chk(cudaMalloc((void**)&L.ring64, sizeof(double) * nring));
      std::vector<int4> dij(goff.size());
      for (size_t q = 0; q < goff.size(); ++q) {
        const int64_t d = goff[q] / L.diamond_stride, r = goff[q] % L.diamond_stride;
        dij[q] = make_int4((int)d, (int)(r / L.P), (int)(r % L.P), 0);
      }
      chk(upload(L.grp_dij, dij));
    }
  }
  chk(cudaMalloc((void**)&L.scr64, sizeof(double) * L.n_layout));
  chk(cudaMalloc((void**)&L.scr32, sizeof(float) * L.n_layout));
  {
    // weight mask (canonical copies), radii, rotation Gram matrix over unique nodes
    std::vector<uint8_t> wm((size_t)L.n_layout, 0);
    const int M = L.N + 1;
    double G[3][3] = {};
    for (int d = 0; d < 10; ++d)
      for (int i = 0; i <= L.N; ++i)
        for (int j = 0; j <= L.N; ++j) {
          const int64_t lat = ((int64_t)d * M + i) * L.P + j;
          if (!owned[lat]) continue;
          const double* s = &L.lat_xyz[(((size_t)d * M + i) * M + j) * 3];
          for (int k = 0; k < L.n_r; ++k) {
            wm[(size_t)(d * L.diamond_stride + k * L.layer_stride + (int64_t)i * L.P + j)] = 1;
            const double r2 = L.radii[k] * L.radii[k];
            for (int a2 = 0; a2 < 3; ++a2)
              for (int b2 = 0; b2 < 3; ++b2) G[a2][b2] += r2 * ((a2 == b2 ? 1.0 : 0.0) - s[a2] * s[b2]);
          }
        }
    std::memcpy(L.inertia, G, sizeof(G));
    chk(upload(L.wmask, wm));
    chk(upload(L.rad64, L.radii));
    chk(upload(L.rad32, to_f32(L.radii)));
  }
  chk(cudaMemset(L.scr64, 0, sizeof(double) * L.n_layout));
  chk(cudaMemset(L.scr32, 0, sizeof(float) * L.n_layout));
  if (e != cudaSuccess) {
    set_error(std::string("tn_mesh_create: device allocation failed: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA;
  }
  return TN_OK;
}

void destroy_level(Level& L) { free_level(L); }

}  // namespace tn

using namespace tn;

extern "C" {

const char* tn_last_error(void) { return g_err.c_str(); }

tn_status tn_mesh_create(int lateral_level, int radial_layers, double r_in, double r_out, const tn_mesh_opts* opts,
                         tn_mesh** out) {
  if (!out) return inval("tn_mesh_create: out is NULL");
  *out = nullptr;
  if (lateral_level < 1 || lateral_level > 12) return inval("tn_mesh_create: lateral_level must be in [1, 12]");
  if (radial_layers < 3 || (radial_layers - 1) % 2 != 0)
    return inval("tn_mesh_create: radial_layers must be >= 3 with radial_layers - 1 even");
  if (!(r_in > 0.0) || !(r_out > r_in)) return inval("tn_mesh_create: need 0 < r_in < r_out");
  tn_mesh_opts o = {TN_BC_FREESLIP, TN_BC_FREESLIP, 1, 0, TN_ETA_F32, 0.0, 1, TN_FP64_ELEM_DOUBLE_FLOAT};
  if (opts) o = *opts;
  if (o.fp64_element != TN_FP64_ELEM_DOUBLE_FLOAT && o.fp64_element != TN_FP64_ELEM_BINARY64)
    return inval("tn_mesh_create: unknown fp64_element");
  if (o.radial_quad_points == 0) o.radial_quad_points = 1;
  if (o.radial_quad_points != 1 && o.radial_quad_points != 2)
    return inval("tn_mesh_create: radial_quad_points must be 1 or 2");
  if (o.eta_storage != TN_ETA_F32 && o.eta_storage != TN_ETA_BF16 && o.eta_storage != TN_ETA_F16)
    return inval("tn_mesh_create: unknown viscosity storage");
  if (!(o.hg_kappa >= 0.0) || o.hg_kappa > 1e6) return inval("tn_mesh_create: hg_kappa must be in [0, 1e6]");
  if (o.radial_quad_points == 2 && o.hg_kappa > 0.0)
    return inval("tn_mesh_create: hourglass control and the second radial point exclude each other");
  if ((o.bc_inner != TN_BC_FREESLIP && o.bc_inner != TN_BC_NOSLIP) ||
      (o.bc_outer != TN_BC_FREESLIP && o.bc_outer != TN_BC_NOSLIP))
    return inval("tn_mesh_create: unknown boundary condition");
  {
    // kernel attributes once per process, before any stream work or graph capture needs them
    static std::once_flag once;
    static cudaError_t prep = cudaSuccess;
    std::call_once(once, [] { prep = prepare_tile_kernels(); });
    if (prep != cudaSuccess) return cuda_fail(prep, "tn_mesh_create: kernel attributes");
  }
  tn_mesh* m = new (std::nothrow) tn_mesh();
  if (!m) {
    set_error("tn_mesh_create: host allocation failed");
    return TN_ENOMEM;
  }
  m->bc_in = o.bc_inner;
  m->bc_out = o.bc_outer;
  m->div_term = o.div_term ? 1 : 0;
  m->eta_storage = o.eta_storage;
  m->hg_kappa = o.hg_kappa;
  m->quad = o.radial_quad_points;
  m->df = o.fp64_element == TN_FP64_ELEM_DOUBLE_FLOAT ? 1 : 0;
  m->r_in = r_in;
  m->r_out = r_out;
  cudaGetDevice(&m->device);
  int l = lateral_level, nr = radial_layers;
  while (true) {
    m->lv.emplace_back();
    tn_status s = create_level(m->lv.back(), l, nr, r_in, r_out, o.eta_storage, m->div_term);
    m->lv.back().hg_kappa = o.hg_kappa;
    m->lv.back().quad = o.radial_quad_points;
    m->lv.back().df = m->df;
    if (s != TN_OK) {
      std::string msg = tn_last_error();
      tn_mesh_destroy(m);
      set_error(msg);
      return s;
    }
    const bool can_coarsen = l >= 2 && (nr - 1) % 2 == 0 && nr >= 3;
    if (!can_coarsen || (o.max_levels > 0 && (int)m->lv.size() >= o.max_levels)) break;
    l -= 1;
    nr = (nr - 1) / 2 + 1;
  }
  *out = m;
  return TN_OK;
}

static void free_step_buffers(tn_mesh* m);

tn_status tn_mesh_destroy(tn_mesh* mesh) {
  if (!mesh) return TN_OK;
  mg_free(mesh->mg);
  mesh->mg = nullptr;
  free_step_buffers(mesh);
  energy_free(mesh);
  for (auto& L : mesh->lv) free_level(L);
  delete mesh;
  return TN_OK;
}

tn_status tn_mesh_info(const tn_mesh* mesh, int level, tn_level_info* info) {
  if (!level_ok(mesh, level) || !info) return inval("tn_mesh_info: bad mesh, level or info");
  const Level& L = mesh->lv[level];
  info->lateral_level = L.l;
  info->N = L.N;
  info->n_r = L.n_r;
  info->pitch = L.P;
  info->layer_stride = L.layer_stride;
  info->diamond_stride = L.diamond_stride;
  info->n_layout = L.n_layout;
  info->n_unique_nodes = ((int64_t)10 * L.N * L.N + 2) * L.n_r;
  info->n_cells = (int64_t)10 * L.N * L.N * (L.n_r - 1);
  info->n_wedges = L.n_wedges;
  info->depth = (int)mesh->lv.size();
  info->r_in = mesh->r_in;
  info->r_out = mesh->r_out;
  return TN_OK;
}

tn_status tn_mesh_lateral_points(const tn_mesh* mesh, int level, double* xyz_host) {
  if (!level_ok(mesh, level) || !xyz_host) return inval("tn_mesh_lateral_points: bad arguments");
  const Level& L = mesh->lv[level];
  std::memcpy(xyz_host, L.lat_xyz.data(), sizeof(double) * L.lat_xyz.size());
  return TN_OK;
}

tn_status tn_mesh_canonical_index(const tn_mesh* mesh, int level, int64_t* canon) {
  if (!level_ok(mesh, level) || !canon) return inval("tn_mesh_canonical_index: bad arguments");
  const Level& L = mesh->lv[level];
  for (int64_t i = 0; i < L.n_layout; ++i) canon[i] = -1;
  for (int d = 0; d < 10; ++d)
    for (int k = 0; k < L.n_r; ++k)
      for (int i = 0; i <= L.N; ++i)
        for (int j = 0; j <= L.N; ++j) {
          int64_t idx = d * L.diamond_stride + k * L.layer_stride + (int64_t)i * L.P + j;
          canon[idx] = idx;
        }
  for (size_t g = 0; g + 1 < L.h_grp_ptr.size(); ++g) {
    int64_t first = L.h_grp_off[L.h_grp_ptr[g]];
    for (int q = L.h_grp_ptr[g]; q < L.h_grp_ptr[g + 1]; ++q)
      for (int k = 0; k < L.n_r; ++k) canon[L.h_grp_off[q] + k * L.layer_stride] = first + k * L.layer_stride;
  }
  return TN_OK;
}

static tn_status finish_eta(tn_mesh* m, cudaStream_t st) {
  for (size_t h = 0; h < m->lv.size(); ++h) {
    if (h > 0) {
      cudaError_t e = launch_eta_coarsen(m->lv[h - 1], m->lv[h], m->lv[h - 1].eta64, m->lv[h].eta64, st);
      if (e != cudaSuccess) return cuda_fail(e, "viscosity coarsening");
    }
    cudaError_t e = launch_eta_f32_path(m->lv[h], st);
    if (e != cudaSuccess) return cuda_fail(e, "viscosity conversion");
  }
  m->eta_set = true;
  mg_invalidate(m);
  return TN_OK;
}

tn_status tn_set_viscosity(tn_mesh* mesh, const double* eta_dev, void* stream) {
  if (!mesh || !eta_dev) return inval("tn_set_viscosity: NULL argument");
  Level& L = mesh->lv[0];
  cudaError_t e = cudaMemcpyAsync(L.eta64, eta_dev, sizeof(double) * L.n_wedges, cudaMemcpyDeviceToDevice, S(stream));
  if (e != cudaSuccess) return cuda_fail(e, "tn_set_viscosity");
  return finish_eta(mesh, S(stream));
}

tn_status tn_set_temperature(tn_mesh* mesh, const double* T_dev, const tn_visc_law* law, void* stream) {
  if (!mesh || !T_dev || !law) return inval("tn_set_temperature: NULL argument");
  Level& L = mesh->lv[0];
  cudaError_t e = launch_eta_from_T(L, T_dev, law->E, law->jump_r, law->jump_factor, L.eta64, S(stream));
  if (e != cudaSuccess) return cuda_fail(e, "tn_set_temperature");
  return finish_eta(mesh, S(stream));
}

tn_status tn_get_viscosity(const tn_mesh* mesh, int level, double* eta_dev, void* stream) {
  if (!level_ok(mesh, level) || !eta_dev) return inval("tn_get_viscosity: bad arguments");
  const Level& L = mesh->lv[level];
  cudaError_t e = cudaMemcpyAsync(eta_dev, L.eta64, sizeof(double) * L.n_wedges, cudaMemcpyDeviceToDevice, S(stream));
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_get_viscosity");
}

static tn_status check_vecs(const char* who, const void* const* a, int na, const void* const* b, int nb) {
  if (!a || !b) return inval(std::string(who) + ": NULL vector array");
  for (int i = 0; i < na; ++i)
    if (!a[i]) return inval(std::string(who) + ": NULL input vector");
  for (int i = 0; i < nb; ++i)
    if (!b[i]) return inval(std::string(who) + ": NULL output vector");
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      if (a[i] == b[j]) return inval(std::string(who) + ": output aliases input");
  for (int i = 0; i < nb; ++i)
    for (int j = i + 1; j < nb; ++j)
      if (b[i] == b[j]) return inval(std::string(who) + ": output components alias each other");
  return TN_OK;
}

tn_status tn_apply_A(tn_mesh* mesh, int level, tn_prec prec, const void* const* u, void* const* y, void* stream) {
  if (!level_ok(mesh, level)) return inval("tn_apply_A: bad mesh or level");
  if (!mesh->eta_set) {
    set_error("tn_apply_A: viscosity not set");
    return TN_ESTATE;
  }
  tn_status s = check_vecs("tn_apply_A", u, 3, (const void* const*)y, 3);
  if (s) return s;
  const Level& L = mesh->lv[level];
  cudaError_t e;
  if (prec == TN_F64)
    e = launch_apply_A<double>(L, bc_of(mesh), mesh->div_term, (const double* const*)u, (double* const*)y, S(stream));
  else if (prec == TN_F32)
    e = launch_apply_A<float>(L, bc_of(mesh), mesh->div_term, (const float* const*)u, (float* const*)y, S(stream));
  else
    return inval("tn_apply_A: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_apply_A");
}

tn_status tn_apply_B(tn_mesh* mesh, int level, tn_prec prec, const void* const* u, void* q, void* stream) {
  if (!level_ok(mesh, level) || level + 1 >= (int)mesh->lv.size()) return inval("tn_apply_B: bad mesh or level");
  void* qa[1] = {q};
  tn_status s = check_vecs("tn_apply_B", u, 3, (const void* const*)qa, 1);
  if (s) return s;
  cudaError_t e;
  if (prec == TN_F64) e = apply_B_t<double>(mesh, level, u, q, S(stream));
  else if (prec == TN_F32) e = apply_B_t<float>(mesh, level, u, q, S(stream));
  else return inval("tn_apply_B: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_apply_B");
}

tn_status tn_apply_BT(tn_mesh* mesh, int level, tn_prec prec, const void* p, void* const* y, void* stream) {
  if (!level_ok(mesh, level) || level + 1 >= (int)mesh->lv.size()) return inval("tn_apply_BT: bad mesh or level");
  const void* pa[1] = {p};
  tn_status s = check_vecs("tn_apply_BT", pa, 1, (const void* const*)y, 3);
  if (s) return s;
  cudaError_t e;
  if (prec == TN_F64) e = apply_BT_t<double>(mesh, level, p, y, S(stream));
  else if (prec == TN_F32) e = apply_BT_t<float>(mesh, level, p, y, S(stream));
  else return inval("tn_apply_BT: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_apply_BT");
}

tn_status tn_diag_A(tn_mesh* mesh, int level, tn_prec prec, void* const* d, void* stream) {
  if (!level_ok(mesh, level)) return inval("tn_diag_A: bad mesh or level");
  if (!mesh->eta_set) {
    set_error("tn_diag_A: viscosity not set");
    return TN_ESTATE;
  }
  const void* none[1] = {nullptr};
  if (!d || !d[0] || !d[1] || !d[2] || d[0] == d[1] || d[0] == d[2] || d[1] == d[2])
    return inval("tn_diag_A: bad output vectors");
  (void)none;
  const Level& L = mesh->lv[level];
  cudaError_t e;
  if (prec == TN_F64) e = launch_diag_A<double>(L, bc_of(mesh), mesh->div_term, (double* const*)d, S(stream));
  else if (prec == TN_F32) e = launch_diag_A<float>(L, bc_of(mesh), mesh->div_term, (float* const*)d, S(stream));
  else return inval("tn_diag_A: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_diag_A");
}

tn_status tn_diag_pmass(tn_mesh* mesh, int level, tn_prec prec, void* m, void* stream) {
  if (!level_ok(mesh, level) || level + 1 >= (int)mesh->lv.size() || !m) return inval("tn_diag_pmass: bad arguments");
  if (!mesh->eta_set) {
    set_error("tn_diag_pmass: viscosity not set");
    return TN_ESTATE;
  }
  cudaError_t e;
  if (prec == TN_F64) e = launch_diag_pmass<double>(mesh->lv[level], mesh->lv[level + 1], (double*)m, S(stream));
  else if (prec == TN_F32) e = launch_diag_pmass<float>(mesh->lv[level], mesh->lv[level + 1], (float*)m, S(stream));
  else return inval("tn_diag_pmass: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_diag_pmass");
}

// ------------------------------------------------------------ operator steps from host memory
static void free_step_buffers(tn_mesh* m) {
  for (auto& set : m->hs_buf)
    for (void*& p : set)
      if (p) {
        cudaFree(p);
        p = nullptr;
      }
  m->hs_elem = 0;
}

// Steps i = 0, 1, ... use buffer set i & 1.  Events order the three streams:
//   copy-in of step i   waits compute of step i - 2 (it overwrites that step's inputs);
//   compute of step i   waits copy-in of step i and copy-out of step i - 2 (it overwrites the
//                       outputs that copy-out reads);
//   copy-out of step i  waits compute of step i.
tn_status tn_operator_steps_host(tn_mesh* mesh, tn_prec prec, int n_steps, const void* const* u_host,
                                 const void* const* p_host, void* const* out_host, void* stream) {
  if (!mesh || mesh->lv.size() < 2) return inval("tn_operator_steps_host: bad mesh (needs a pressure level)");
  if (prec != TN_F64 && prec != TN_F32) return inval("tn_operator_steps_host: unknown precision");
  if (n_steps < 0) return inval("tn_operator_steps_host: n_steps < 0");
  if (n_steps > 0 && (!u_host || !p_host || !out_host)) return inval("tn_operator_steps_host: NULL pointer array");
  for (int i = 0; i < n_steps; ++i) {
    if (!u_host[3 * i] || !u_host[3 * i + 1] || !u_host[3 * i + 2] || !p_host[i])
      return inval("tn_operator_steps_host: NULL input buffer");
    for (int k = 0; k < 10; ++k)
      if (!out_host[10 * i + k]) return inval("tn_operator_steps_host: NULL output buffer");
  }
  if (!mesh->eta_set) {
    set_error("tn_operator_steps_host: viscosity not set");
    return TN_ESTATE;
  }
  if (n_steps == 0) return TN_OK;
  const size_t es = prec == TN_F64 ? sizeof(double) : sizeof(float);
  const int64_t n0 = mesh->lv[0].n_layout, n1 = mesh->lv[1].n_layout;
  const int64_t len[14] = {n0, n0, n0, n1, n0, n0, n0, n1, n0, n0, n0, n0, n0, n0};
  if (mesh->hs_elem != es) {
    free_step_buffers(mesh);
    for (auto& set : mesh->hs_buf)
      for (int v = 0; v < 14; ++v)
        // zeroed once: the layout's padding entries, which no kernel writes, read back as 0
        if (cudaMalloc(&set[v], es * len[v]) != cudaSuccess || cudaMemset(set[v], 0, es * len[v]) != cudaSuccess) {
          cudaGetLastError();
          free_step_buffers(mesh);
          set_error("tn_operator_steps_host: device buffers");
          return TN_ENOMEM;
        }
    mesh->hs_elem = es;
  }
  const cudaStream_t cs = S(stream);
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr, ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    e = cudaEventCreateWithFlags(&ev_in[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_comp[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[s], cudaEventDisableTiming);
  }
  tn_status st = TN_OK;
  if (e == cudaSuccess) e = cudaEventRecord(start, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h2d, start, 0);
  for (int i = 0; i < n_steps && e == cudaSuccess && st == TN_OK; ++i) {
    const int s = i & 1;
    void* const* B = mesh->hs_buf[s];
    if (i >= 2) e = cudaStreamWaitEvent(h2d, ev_comp[s], 0);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c)
      e = cudaMemcpyAsync(B[c], u_host[3 * i + c], es * n0, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B[3], p_host[i], es * n1, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[s], h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in[s], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(cs, ev_out[s], 0);
    if (e != cudaSuccess) break;
    const void* u[3] = {B[0], B[1], B[2]};
    void* yA[3] = {B[4], B[5], B[6]};
    void* yBT[3] = {B[8], B[9], B[10]};
    void* d[3] = {B[11], B[12], B[13]};
    st = tn_apply_A(mesh, 0, prec, u, yA, stream);
    if (st == TN_OK) st = tn_apply_B(mesh, 0, prec, u, B[7], stream);
    if (st == TN_OK) st = tn_apply_BT(mesh, 0, prec, B[3], yBT, stream);
    if (st == TN_OK) st = tn_diag_A(mesh, 0, prec, d, stream);
    if (st != TN_OK) break;
    e = cudaEventRecord(ev_comp[s], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, ev_comp[s], 0);
    for (int k = 0; k < 10 && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(out_host[10 * i + k], B[4 + k], es * len[4 + k], cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[s], d2h);
  }
  // `stream` waits for everything enqueued on the two private streams -- after an early exit too,
  // so that no copy into the mesh's buffers outlives the caller's stream order (a retry on the same
  // mesh would otherwise overlap it); if the join itself fails, the host waits instead
  for (cudaStream_t x : {h2d, d2h}) {
    if (!x) continue;
    cudaEvent_t tail = nullptr;
    cudaError_t w = cudaEventCreateWithFlags(&tail, cudaEventDisableTiming);
    if (w == cudaSuccess) w = cudaEventRecord(tail, x);
    if (w == cudaSuccess) w = cudaStreamWaitEvent(cs, tail, 0);
    if (tail) cudaEventDestroy(tail);
    if (w != cudaSuccess) {
      cudaStreamSynchronize(x);
      if (e == cudaSuccess) e = w;
    }
  }
  // destruction is deferred by the runtime until the enqueued work is complete
  cudaEvent_t evs[7] = {start, ev_in[0], ev_in[1], ev_comp[0], ev_comp[1], ev_out[0], ev_out[1]};
  for (cudaEvent_t x : evs)
    if (x) cudaEventDestroy(x);
  if (h2d) cudaStreamDestroy(h2d);
  if (d2h) cudaStreamDestroy(d2h);
  if (st != TN_OK) return st;
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_operator_steps_host");
}

tn_status tn_prolong(tn_mesh* mesh, int level, tn_prec prec, int ncomp, int apply_bc, const void* const* c,
                     void* const* f, void* stream) {
  if (!level_ok(mesh, level) || level + 1 >= (int)mesh->lv.size()) return inval("tn_prolong: bad mesh or level");
  if (ncomp != 1 && ncomp != 3) return inval("tn_prolong: ncomp must be 1 or 3");
  tn_status s = check_vecs("tn_prolong", c, ncomp, (const void* const*)f, ncomp);
  if (s) return s;
  const Level& F = mesh->lv[level];
  const Level& C = mesh->lv[level + 1];
  cudaError_t e;
  if (prec == TN_F64)
    e = launch_prolong<double>(F, C, bc_of(mesh), ncomp, apply_bc, (const double* const*)c, (double* const*)f, S(stream));
  else if (prec == TN_F32)
    e = launch_prolong<float>(F, C, bc_of(mesh), ncomp, apply_bc, (const float* const*)c, (float* const*)f, S(stream));
  else return inval("tn_prolong: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_prolong");
}

tn_status tn_restrict(tn_mesh* mesh, int level, tn_prec prec, int ncomp, int apply_bc, const void* const* f,
                      void* const* c, void* stream) {
  if (!level_ok(mesh, level) || level + 1 >= (int)mesh->lv.size()) return inval("tn_restrict: bad mesh or level");
  if (ncomp != 1 && ncomp != 3) return inval("tn_restrict: ncomp must be 1 or 3");
  tn_status s = check_vecs("tn_restrict", f, ncomp, (const void* const*)c, ncomp);
  if (s) return s;
  const Level& F = mesh->lv[level];
  const Level& C = mesh->lv[level + 1];
  cudaError_t e;
  if (prec == TN_F64)
    e = launch_restrict<double>(F, C, bc_of(mesh), ncomp, apply_bc, (const double* const*)f, (double* const*)c, S(stream));
  else if (prec == TN_F32)
    e = launch_restrict<float>(F, C, bc_of(mesh), ncomp, apply_bc, (const float* const*)f, (float* const*)c, S(stream));
  else return inval("tn_restrict: unknown precision");
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_restrict");
}

tn_status tn_set_reference_state(tn_mesh* mesh, const double* rho_host, const double* alpha_host) {
  if (!mesh) return inval("tn_set_reference_state: NULL mesh");
  Level& L = mesh->lv[0];
  const int nr = L.n_r;
  std::vector<double> rho, alpha(nr, 1.0), bw(nr - 1);
  if (rho_host) {
    rho.assign(rho_host, rho_host + nr);
    if (alpha_host) alpha.assign(alpha_host, alpha_host + nr);
    for (int k = 0; k < nr; ++k)
      if (!(rho[k] > 0.0) || !std::isfinite(rho[k]) || !std::isfinite(alpha[k]))
        return inval("tn_set_reference_state: rho must be positive and finite, alpha finite");
  }
  // layer-table slots 10, 11: rho(q_c) and rho'(q_c) / (6 w0) (zero without a reference state)
  std::vector<double> lay = L.h_lay;
  for (int k = 0; k + 1 < nr; ++k) {
    double* t = &lay[(size_t)kLayerStride * k];
    if (rho_host) {
      const double w0 = t[0];
      t[10] = 0.5 * (rho[k] + rho[k + 1]);
      t[11] = (rho[k + 1] - rho[k]) / (L.radii[k + 1] - L.radii[k]) / (6.0 * w0);
      bw[k] = (0.5 * (rho[k] + rho[k + 1])) * (0.5 * (alpha[k] + alpha[k + 1]));
    } else {
      t[10] = t[11] = 0.0;
    }
  }
  const std::vector<float> l32 = to_f32(lay), ldf = to_df(lay);
  cudaError_t e = cudaMemcpy(L.lay64, lay.data(), sizeof(double) * lay.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L.lay32, l32.data(), sizeof(float) * l32.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L.laydf, ldf.data(), sizeof(float) * ldf.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && rho_host && !L.bw64) e = cudaMalloc((void**)&L.bw64, sizeof(double) * (nr - 1));
  if (e == cudaSuccess && rho_host)
    e = cudaMemcpy(L.bw64, bw.data(), sizeof(double) * (nr - 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "tn_set_reference_state");
  if (!rho_host && L.bw64) {
    cudaFree(L.bw64);
    L.bw64 = nullptr;
  }
  L.h_lay = lay;
  L.tala = rho_host ? 1 : 0;
  mg_invalidate(mesh);  // the Schur deflation vector of the solver depends on B
  return TN_OK;
}

tn_status tn_buoyancy(tn_mesh* mesh, const double* T_dev, double Ra, double* const* f, void* stream) {
  if (!mesh || !T_dev || !f || !f[0] || !f[1] || !f[2]) return inval("tn_buoyancy: NULL argument");
  cudaError_t e = launch_buoyancy(mesh->lv[0], bc_of(mesh), T_dev, Ra, f, S(stream));
  return e == cudaSuccess ? TN_OK : cuda_fail(e, "tn_buoyancy");
}

}  // extern "C"
