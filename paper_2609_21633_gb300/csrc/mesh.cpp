// Host construction of one level of the icosahedral shell (paper Sec. 2, Fig. 1).
//
// Compiled with -ffp-contract=off: every value below is a fixed sequence of
// IEEE operations, so x86 and Arm hosts produce identical tables, and the
// copies of a diamond-edge point generated in different diamonds coincide
// bitwise (they are normalised sums of the same end points).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "internal.h"

namespace tn {

namespace {

using V3 = std::array<double, 3>;

V3 normalized_sum(const V3& p, const V3& q) {
  V3 v = {p[0] + q[0], p[1] + q[1], p[2] + q[2]};
  double n = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  return {v[0] / n, v[1] / n, v[2] / n};
}

// 12 icosahedron vertices: N pole, upper ring U_k (latitude +atan(1/2), longitude 72k deg),
// lower ring L_k (latitude -atan(1/2), longitude 36 + 72k deg), S pole.
void icosahedron(V3& north, V3& south, V3 up[5], V3 lo[5]) {
  const double pi = 3.14159265358979323846;
  double lat = std::atan(0.5);
  north = {0.0, 0.0, 1.0};
  south = {0.0, 0.0, -1.0};
  for (int k = 0; k < 5; ++k) {
    double lu = 2.0 * pi * k / 5.0;
    double ll = pi / 5.0 + 2.0 * pi * k / 5.0;
    up[k] = {std::cos(lat) * std::cos(lu), std::cos(lat) * std::sin(lu), std::sin(lat)};
    lo[k] = {std::cos(-lat) * std::cos(ll), std::cos(-lat) * std::sin(ll), std::sin(-lat)};
  }
}

}  // namespace

void build_lateral_points(int level, std::vector<double>& pts) {
  const int N = 1 << level, M = N + 1;
  pts.assign((size_t)10 * M * M * 3, 0.0);
  V3 north, south, up[5], lo[5];
  icosahedron(north, south, up, lo);
  auto at = [&](int d, int i, int j) -> double* { return &pts[(((size_t)d * M + i) * M + j) * 3]; };
  auto get = [&](int d, int i, int j) {
    double* p = at(d, i, j);
    return V3{p[0], p[1], p[2]};
  };
  auto put = [&](int d, int i, int j, const V3& v) {
    double* p = at(d, i, j);
    p[0] = v[0], p[1] = v[1], p[2] = v[2];
  };
  for (int k = 0; k < 5; ++k) {
    int k1 = (k + 1) % 5;
    // diamond corners (c00, c10, c01, c11) = lattice (0,0), (N,0), (0,N), (N,N)
    put(k, 0, 0, north), put(k, N, 0, up[k]), put(k, 0, N, up[k1]), put(k, N, N, lo[k]);
    put(5 + k, 0, 0, up[k1]), put(5 + k, N, 0, lo[k]), put(5 + k, 0, N, lo[k1]), put(5 + k, N, N, south);
  }
  for (int s = N; s > 1; s /= 2) {
    const int h = s / 2;
    for (int d = 0; d < 10; ++d) {
      for (int i = 0; i + s <= N; i += s)
        for (int j = 0; j <= N; j += s) put(d, i + h, j, normalized_sum(get(d, i, j), get(d, i + s, j)));
      for (int i = 0; i <= N; i += s)
        for (int j = 0; j + s <= N; j += s) put(d, i, j + h, normalized_sum(get(d, i, j), get(d, i, j + s)));
      for (int i = 0; i + s <= N; i += s)
        for (int j = 0; j + s <= N; j += s)
          put(d, i + h, j + h, normalized_sum(get(d, i + s, j), get(d, i, j + s)));
    }
  }
}

void build_level_host(Level& L, int level, int n_r, double r_in, double r_out, std::vector<double>& geo,
                      std::vector<double>& lay, std::vector<double>& s, std::vector<int>& grp_ptr,
                      std::vector<int64_t>& grp_off, std::vector<double>& grp_s, std::vector<uint8_t>& owned,
                      std::string& err) {
  const int N = 1 << level, M = N + 1;
  L.l = level;
  L.N = N;
  L.n_r = n_r;
  L.P = (M + 3) / 4 * 4;
  L.layer_stride = (int64_t)M * L.P;
  L.diamond_stride = (int64_t)n_r * L.layer_stride;
  L.n_layout = 10 * L.diamond_stride;
  L.n_tri = (int64_t)10 * N * N * 2;
  L.n_wedges = L.n_tri * (n_r - 1);
  L.n_lat_layout = (int64_t)10 * M * L.P;
  build_lateral_points(level, L.lat_xyz);
  L.radii.resize(n_r);
  for (int k = 0; k < n_r; ++k) L.radii[k] = r_in + ((r_out - r_in) * k) / (n_r - 1);

  auto S = [&](int d, int i, int j, int c) { return L.lat_xyz[(((size_t)d * M + i) * M + j) * 3 + c]; };

  // ---- per-triangle geometry: M = [s1 - s0, s2 - s0, sbar] (columns), J = M diag(rho, rho, h)
  geo.assign((size_t)10 * L.n_tri, 0.0);
  for (int d = 0; d < 10; ++d)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int w = 0; w < 2; ++w) {
          int pi_[3], pj_[3];
          if (w == 0) {
            pi_[0] = i, pj_[0] = j, pi_[1] = i + 1, pj_[1] = j, pi_[2] = i, pj_[2] = j + 1;
          } else {
            pi_[0] = i + 1, pj_[0] = j + 1, pi_[1] = i, pj_[1] = j + 1, pi_[2] = i + 1, pj_[2] = j;
          }
          double m[3][3];  // m[x][col]
          for (int x = 0; x < 3; ++x) {
            double s0 = S(d, pi_[0], pj_[0], x), s1 = S(d, pi_[1], pj_[1], x), s2 = S(d, pi_[2], pj_[2], x);
            m[x][0] = s1 - s0;
            m[x][1] = s2 - s0;
            m[x][2] = (s0 + s1 + s2) / 3.0;
          }
          double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
          double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
          double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
          double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
          double inv[3][3];  // inv[col][x] = (M^{-1})[col][x]
          inv[0][0] = c00 / det;
          inv[1][0] = c01 / det;
          inv[2][0] = c02 / det;
          inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
          inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
          inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
          inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
          inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
          inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
          int64_t t = (((int64_t)d * N + i) * N + j) * 2 + w;
          for (int a = 0; a < 3; ++a)
            for (int x = 0; x < 3; ++x) geo[(size_t)(a * 3 + x) * L.n_tri + t] = inv[a][x];
          geo[(size_t)9 * L.n_tri + t] = std::fabs(det);
          if (!(det > 0.0)) err = "degenerate or inverted lateral triangle";
        }

  // ---- per radial cell: (w0, w1, vol, rho, w1 / w0, vol w0^2, vol w0, -vol w0 / 6,
  // w0 / (9 w1), vol w1^2, 0, 0) with w0 = 1/(2 rho), w1 = 1/(6 h), vol = rho^2 h
  lay.assign((size_t)kLayerStride * (n_r - 1), 0.0);
  for (int k = 0; k + 1 < n_r; ++k) {
    double rho = 0.5 * (L.radii[k] + L.radii[k + 1]);
    double h = 0.5 * (L.radii[k + 1] - L.radii[k]);
    double* t = &lay[(size_t)kLayerStride * k];
    t[0] = 1.0 / (2.0 * rho);
    t[1] = 1.0 / (6.0 * h);
    t[2] = rho * rho * h;
    t[3] = rho;
    t[4] = t[1] / t[0];
    t[5] = t[2] * t[0] * t[0];
    t[6] = t[2] * t[0];
    t[7] = -t[6] / 6.0;
    t[8] = t[0] / (9.0 * t[1]);
    t[9] = t[2] * t[1] * t[1];
  }

  // ---- lateral unit vectors in the padded lateral layout
  s.assign((size_t)3 * L.n_lat_layout, 0.0);
  for (int d = 0; d < 10; ++d)
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N; ++j)
        for (int c = 0; c < 3; ++c)
          s[(size_t)c * L.n_lat_layout + ((int64_t)d * M + i) * L.P + j] = S(d, i, j, c);

  // ---- interface groups: lattice points on diamond edges, grouped by exact coordinates
  struct Key {
    uint64_t b[3];
    bool operator<(const Key& o) const {
      return b[0] != o.b[0] ? b[0] < o.b[0] : (b[1] != o.b[1] ? b[1] < o.b[1] : b[2] < o.b[2]);
    }
  };
  std::map<Key, std::vector<int64_t>> groups;
  std::map<Key, V3> gpos;
  for (int d = 0; d < 10; ++d)
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N; ++j) {
        if (!(i == 0 || i == N || j == 0 || j == N)) continue;
        Key key;
        V3 p = {S(d, i, j, 0), S(d, i, j, 1), S(d, i, j, 2)};
        for (int c = 0; c < 3; ++c) std::memcpy(&key.b[c], &p[c], 8);
        groups[key].push_back((int64_t)d * L.diamond_stride + (int64_t)i * L.P + j);
        gpos[key] = p;
      }
  grp_ptr.assign(1, 0);
  grp_off.clear();
  std::vector<V3> gs;
  int n2 = 0, n3 = 0, n5 = 0;
  owned.assign((size_t)L.n_lat_layout, 0);
  for (int d = 0; d < 10; ++d)
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N; ++j) owned[((int64_t)d * M + i) * L.P + j] = 1;
  // groups in layout order of their first copy, so that neighbouring groups along a diamond row
  // are neighbouring threads of the interface kernels (coalesced accesses)
  std::vector<std::pair<int64_t, const Key*>> order;
  for (auto& kv : groups) {
    std::sort(kv.second.begin(), kv.second.end());
    order.push_back({kv.second[0], &kv.first});
  }
  std::sort(order.begin(), order.end());
  for (auto& ok : order) {
    auto& v = groups[*ok.second];
    if (v.size() == 2) ++n2;
    else if (v.size() == 3) ++n3;
    else if (v.size() == 5) ++n5;
    else {
      err = "interface group of unexpected size";
      continue;
    }
    for (size_t c = 1; c < v.size(); ++c) {
      int64_t off = v[c];
      int64_t d = off / L.diamond_stride, rem = off % L.diamond_stride;
      owned[d * M * L.P + rem] = 0;
    }
    grp_off.insert(grp_off.end(), v.begin(), v.end());
    grp_ptr.push_back((int)grp_off.size());
    gs.push_back(gpos[*ok.second]);
  }
  if (n2 != 20 * (N - 1) || n3 != 10 || n5 != 2) err = "interface groups do not match the icosahedral topology";
  L.n_groups = (int)gs.size();
  grp_s.assign((size_t)3 * L.n_groups, 0.0);
  for (int g = 0; g < L.n_groups; ++g)
    for (int c = 0; c < 3; ++c) grp_s[(size_t)c * L.n_groups + g] = gs[g][c];
}

}  // namespace tn
