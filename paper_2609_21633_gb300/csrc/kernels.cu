// sm_103a kernels of the matrix-free wedge Stokes operator.
//
// Element-level work follows Eq. (epsq) / Eq. (localapply) with one quadrature
// point at the wedge barycentre q_c (Sec. 4): the strain of the gathered
// element DoFs is formed at q_c, contracted into the stress, and the stress is
// contracted with every test gradient -- the 18 x 18 element matrix is never
// formed (Sec. 6).  Geometry is factorised: at q_c the isoparametric Jacobian
// of a wedge between radii r_k and r_k+1 over lateral unit vectors s0, s1, s2
// is J = M diag(rho, rho, h), M = [s1 - s0, s2 - s0, (s0 + s1 + s2)/3],
// rho = (r_k + r_k+1)/2, h = (r_k+1 - r_k)/2, so a lateral table of M^{-1}
// and |det M| plus a per-layer table of (1/(2 rho), 1/(6 h), rho^2 h) carry
// all of it ("radial coordinate compression").  With g'_j the reference
// gradients scaled to entries in {-1, 0, 1}:
//     grad u  = sum_m a_m W_m M^{-1}[m, :],   a_m = sum_j u_j g'_j[m]
//     y_j     = sum_m g'_j[m] H[:, m],        H[:, m] = W_m S M^{-1}[m, :]^T
// with W = (1/(2 rho), 1/(2 rho), 1/(6 h)) and S = V eta (grad u + grad u^T
// - 2/3 tr(grad u) I) the stress of Eq. (stress) times V = rho^2 h |det M|.
//
// The element-to-node scatter is deterministic and atomic-free: a CTA owns a
// tile of lateral node columns, computes every cell that touches it (one
// halo cell row / column), and streams the radial direction, carrying each
// cell's top-face contributions in registers to the next layer.  Lateral
// contributions of the four cells around a node are exchanged through shared
// memory and summed in a fixed order.  Nodes on diamond edges receive a
// partial sum per diamond; launch_interface adds the copies in ascending
// layout order and writes the total to every copy (the on-device stand-in
// for the paper's additive halo exchange, Sec. 2).
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dfloat.cuh"
#include "internal.h"

// The file is compiled five times: TN_PART 1 holds everything but the A-apply launchers, TN_PART 2
// the FP64 and TN_PART 3 the FP32 A-apply launchers, TN_PART 4 and 5 those of the A apply with
// the second radial quadrature point (their many tile-kernel instantiations then compile in
// parallel); 0 = all.
#ifndef TN_PART
#define TN_PART 0
#endif

namespace tn {

namespace {

constexpr int TILE = 16;  // lateral nodes per tile edge (N >= 16), else N

inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Resident CTAs per SM requested from the register allocator for the tile kernel, per precision.
#ifndef TN_MINB_F64
#define TN_MINB_F64 2
#endif
#ifndef TN_MINB_F32
#define TN_MINB_F32 2
#endif
// Radial chunking: the grid is split radially until it has at least this many CTAs
// (chunks never shorter than TN_KC_MIN cells).
#ifndef TN_CTA_TARGET
#define TN_CTA_TARGET (32 * 152)
#endif
// CTA target for wide (16 x 32) tiles, which run one CTA per SM; 0 disables wide tiles.
#ifndef TN_CTA_TARGET_WIDE
#define TN_CTA_TARGET_WIDE (16 * 152)
#endif
#ifndef TN_WIDE_TILES
#define TN_WIDE_TILES 1
#endif
// 1: FP64 levels with N >= 32 use halo-free 16 x 32 tiles plus the tile-line pass
#ifndef TN_HALO_FREE
#define TN_HALO_FREE 1
#endif
// 1: the epilogue variants prefetch their per-node operands before the cell arithmetic
#ifndef TN_EPI_PREFETCH
#define TN_EPI_PREFETCH 1
#endif
// Register cap of the wide tiles: 561 threads are 18 warps, allocated as 20 (a multiple of the 4
// sub-partitions), so 65536 / (20 x 32) rounds down to 96 registers per thread.
#ifndef TN_WIDE_MAXREG
#define TN_WIDE_MAXREG 96
#endif
#ifndef TN_KC_MIN
#define TN_KC_MIN 8
#endif
// 1: load node layer k+2 while cell layer k is computed
#ifndef TN_PREFETCH
#define TN_PREFETCH 0
#endif
// FP32 A apply on paired-cell tiles (pair32.cuh) where N >= 32 (0: the square tiles), and its CTA
// target: radial chunks halve until the grid has this many CTAs (two resident per SM)
#ifndef TN_PAIR32
#define TN_PAIR32 1
#endif
#ifndef TN_PAIR_CTA_TARGET
#define TN_PAIR_CTA_TARGET (16 * 152)
#endif
template <typename T>
struct MinBlocks {
  static constexpr int value = sizeof(T) == 8 ? TN_MINB_F64 : TN_MINB_F32;
};

template <typename T>
struct Tab;  // precision-selected views of a level's tables
template <>
struct Tab<double> {
  static const double* geo(const Level& L) { return L.geo64; }
  static const double* lay(const Level& L) { return L.lay64; }
  static const double* s(const Level& L) { return L.s64; }
  static const double* gs(const Level& L) { return L.grp_s64; }
  static const double* dcoef(const Level& L) { return L.dcoef64; }
};
template <>
struct Tab<float> {
  static const float* geo(const Level& L) { return L.geo32; }
  static const float* lay(const Level& L) { return L.lay32; }
  static const float* s(const Level& L) { return L.s32; }
  static const float* gs(const Level& L) { return L.grp_s32; }
  static const float* dcoef(const Level& L) { return L.dcoef32; }
};

// Per-wedge viscosity as a kernel reads it: v[w] (kind TN_ETA_F32, and always for FP64), or
// the 16-bit q[w] times the column factor cs[t] of lateral wedge t (kinds TN_ETA_BF16 / F16).
template <typename T>
struct EtaView {
  const T* v;
  const uint16_t* q;
  const float* cs;
  int kind;
};
inline EtaView<double> eta_view(const Level& L, double*) { return EtaView<double>{L.eta64, nullptr, nullptr, 0}; }
inline EtaView<float> eta_view(const Level& L, float*) {
  return EtaView<float>{L.eta32, L.eta16, L.eta_cs, L.eta_kind};
}
template <typename T>
EtaView<T> etav(const Level& L) {
  return eta_view(L, (T*)nullptr);
}

template <int KIND>
__device__ __forceinline__ float from16(uint16_t b) {
  if (KIND == TN_ETA_BF16) return __bfloat162float(__ushort_as_bfloat16(b));
  return __half2float(__ushort_as_half(b));
}

// Viscosity of wedge index w in lateral column t (kind chosen at run time).
template <typename T>
__device__ __forceinline__ T eta_at(const EtaView<T>& E, int64_t w, int64_t t) {
  if (E.kind == TN_ETA_F32) return E.v[w];
  const float f = E.kind == TN_ETA_BF16 ? from16<TN_ETA_BF16>(E.q[w]) : from16<TN_ETA_F16>(E.q[w]);
  return (T)(f * E.cs[t]);
}


// ------------------------------------------------------------------------------------ element ops
// An op processes both wedges of one hexahedral cell.  Inputs are, at the cell's four lateral
// corners (00, 10, 01, 11), the sums s = top + bottom and differences d = top - bottom of the
// nodal values on its bottom and top node layer (computed once per node by the tile kernel);
// the op assigns the cell's contributions to the same eight node slots (accb, acct), every
// entry.  Wedge-local lateral node a of wedge w sits at corner kCorner[w][a]: W0 = (00, 10, 01),
// W1 = (11, 01, 10), so corner 00 belongs to W0 only, 11 to W1 only and 10, 01 to both.  `lc`
// points at the cell layer's table entry (w0, w1, vol, rho, r = w1 / w0, vol w0^2, vol w0,
// -vol w0 / 6).
//
// With a_xi = s_c1 - s_c0, a_eta = s_c2 - s_c0, a_zeta = d_c0 + d_c1 + d_c2 (s = top + bottom,
// d = top - bottom, per component; the reference gradients scaled to {-1, 0, 1}), the strain
// G' = a_xi M^-1[0,:] + a_eta M^-1[1,:] + a_zeta r M^-1[2,:] is grad u / w0, and
// S'' = vol w0^2 |det M| eta (G' + G'^T - 2/3 tr G' I) is the stress of Eq. (stress) times
// V w0.  Then H[:,0] = S'' M^-1[0,:]^T, H[:,1] = S'' M^-1[1,:]^T, H[:,2] = S'' r M^-1[2,:]^T
// and node (a, bottom / top) receives X_a -/+ H[:,2], X = (-H[:,0] - H[:,1], H[:,0], H[:,1]).
// Contributions are assigned where a corner is first touched and added otherwise (adding to a
// zero start would cost an instruction per entry: x + 0 cannot be folded in IEEE arithmetic).
__device__ constexpr int kCorner[2][3] = {{0, 1, 2}, {3, 2, 1}};

// Corner combination shared by the vector-valued ops: X[q] are the per-corner sums of X, h[w]
// the H[:,2] column of wedge w; corner 00 gets h[0], 11 gets h[1], 10 and 01 get both.
template <typename T, int NC>
__device__ __forceinline__ void combine_corners(const T (&X)[4][NC], const T (&h)[2][NC], T (&accb)[4][NC],
                                                T (&acct)[4][NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T h01 = h[0][c] + h[1][c];
    accb[0][c] = X[0][c] - h[0][c], acct[0][c] = X[0][c] + h[0][c];
    accb[3][c] = X[3][c] - h[1][c], acct[3][c] = X[3][c] + h[1][c];
    accb[1][c] = X[1][c] - h01, acct[1][c] = X[1][c] + h01;
    accb[2][c] = X[2][c] - h01, acct[2][c] = X[2][c] + h01;
  }
}

// Per-column state of the ops without any: nothing.
struct NoCol {};

// Hourglass control, Eq. (hgstab), in the scaled quantities above.  With the hourglass vectors
// made orthogonal to the physical linear fields (g_m = w_m - sum_c (w_m . X_c) dN/dx_c), and
// w_1 . X = 2h (s_1 - sbar), w_2 . X = 2h (s_2 - sbar), (s_a - sbar) . M^-1[m,:] known from
// M^-1 M = I, everything reduces to k9 = w0 / (9 w1) = 1 / (9 r):
//   alpha_1 = g_1 . u = (d_c1 - a_zeta / 3) - k9 (2 a_xi - a_eta),
//   alpha_2 = g_2 . u = (d_c2 - a_zeta / 3) - k9 (2 a_eta - a_xi),
// and eps sum_m alpha_m g_m adds -eps k9 b_1 to H[:,0], -eps k9 b_2 to H[:,1] and
// +/- eps / 3 (-(b_1 + b_2), b_1, b_2) at lateral nodes (a = 0, 1, 2) on the top / bottom layer,
// b_1 = 2 alpha_1 - alpha_2, b_2 = 2 alpha_2 - alpha_1.  eps = hgk eta (vol w0^2 eL + vol w1^2 eR),
// hgk = kappa (3 + c) / 18, eL = 2 |det M| (|m0 + m1|^2 + |m0|^2 + |m1|^2), eR = 6 |det M| |m2|^2
// (m = rows of M^-1): kappa tr(A_e) / 18, since tr(A_e) = V eta (3 + c) sum_j |grad N_j|^2.
template <typename T>
struct HgCol {
  T eL[2], eR[2];
};
template <typename T>
__device__ __forceinline__ HgCol<T> hg_column(const T (&Mi)[2][9], const T (&dM)[2]) {
  HgCol<T> col;
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    const T* M = Mi[w];
    T l = 0, q = 0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const T s01 = M[x] + M[3 + x];
      l += s01 * s01 + M[x] * M[x] + M[3 + x] * M[3 + x];
      q += M[6 + x] * M[6 + x];
    }
    col.eL[w] = (T)2 * dM[w] * l;
    col.eR[w] = (T)6 * dM[w] * q;
  }
  return col;
}

// Viscous block: Eq. (epsq) then Eq. (localapply) at q_c; HG adds the hourglass control.
template <typename T, bool HG = false>
struct OpA {
  static constexpr int NIN = 3, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = true, NEEDS_D = true;
  using Col = typename std::conditional<HG, HgCol<T>, NoCol>::type;
  int div_term;
  T hgk;  // kappa (3 + c) / 18 (HG only)
  __device__ __forceinline__ Col column(const T (&Mi)[2][9], const T (&dM)[2], int) const {
    if constexpr (HG) return hg_column(Mi, dM);
    else return Col{};
  }
  __device__ __forceinline__ void cell(const T (&s)[4][3], const T (&dd)[4][3], const T (&Mi)[2][9],
                                       const T (&dM)[2], const T* lc, const T (&eta)[2], T (&accb)[4][3],
                                       T (&acct)[4][3], const Col& col) const {
    const T r = lc[4], vw2 = lc[5];
    // X: per-corner sums of X; without HG h[w] is the H[:,2] column of wedge w, with HG Y holds
    // the per-corner sums of the top-minus-bottom part
    T X[4][3], h[2][3], Y[4][3];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int c0 = kCorner[w][0], c1 = kCorner[w][1], c2 = kCorner[w][2];
      const T* M = Mi[w];
      const T mr[3] = {r * M[6], r * M[7], r * M[8]};  // r M^-1[2,:]
      T G[3][3], al1[3], al2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T ax = s[c1][c] - s[c0][c], ay = s[c2][c] - s[c0][c], az = (dd[c0][c] + dd[c1][c]) + dd[c2][c];
#pragma unroll
        for (int x = 0; x < 3; ++x) G[c][x] = ax * M[x] + ay * M[3 + x] + az * mr[x];
        if constexpr (HG) {
          const T k9 = lc[8], a3 = az * (T)(1.0 / 3.0);
          al1[c] = (dd[c1][c] - a3) - k9 * (ax + ax - ay);
          al2[c] = (dd[c2][c] - a3) - k9 * (ay + ay - ax);
        }
      }
      const T ve = vw2 * dM[w] * eta[w];
      const T ve2 = ve + ve;
      T S[3][3];
      if (div_term) {
        const T vt = (ve * (T)(-2.0 / 3.0)) * ((G[0][0] + G[1][1]) + G[2][2]);
        S[0][0] = ve2 * G[0][0] + vt, S[1][1] = ve2 * G[1][1] + vt, S[2][2] = ve2 * G[2][2] + vt;
      } else {
        S[0][0] = ve2 * G[0][0], S[1][1] = ve2 * G[1][1], S[2][2] = ve2 * G[2][2];
      }
      S[0][1] = S[1][0] = ve * (G[0][1] + G[1][0]);
      S[0][2] = S[2][0] = ve * (G[0][2] + G[2][0]);
      S[1][2] = S[2][1] = ve * (G[1][2] + G[2][1]);
      T ek = 0, e3 = 0;
      if constexpr (HG) {
        const T eps = (hgk * eta[w]) * (vw2 * col.eL[w] + lc[9] * col.eR[w]);
        ek = eps * lc[8], e3 = eps * (T)(1.0 / 3.0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T h0 = S[c][0] * M[0] + S[c][1] * M[1] + S[c][2] * M[2];
        T h1 = S[c][0] * M[3] + S[c][1] * M[4] + S[c][2] * M[5];
        const T h2 = S[c][0] * mr[0] + S[c][1] * mr[1] + S[c][2] * mr[2];
        if constexpr (HG) {
          const T b1 = (al1[c] + al1[c]) - al2[c], b2 = (al2[c] + al2[c]) - al1[c];
          h0 -= ek * b1, h1 -= ek * b2;
          const T v1 = e3 * b1, v2 = e3 * b2;
          const T y0 = h2 - (v1 + v2), y1 = h2 + v1, y2 = h2 + v2;
          Y[c0][c] = y0;
          if (w == 0) {
            Y[c1][c] = y1, Y[c2][c] = y2;
          } else {
            Y[c1][c] += y1, Y[c2][c] += y2;
          }
        } else {
          h[w][c] = h2;
        }
        X[c0][c] = -(h0 + h1);
        if (w == 0) {
          X[c1][c] = h0, X[c2][c] = h1;
        } else {
          X[c1][c] += h0, X[c2][c] += h1;
        }
      }
    }
    if constexpr (HG) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) accb[q][c] = X[q][c] - Y[q][c], acct[q][c] = X[q][c] + Y[q][c];
    } else {
      combine_corners<T, 3>(X, h, accb, acct);
    }
  }
};

// Double-float viscous block without hourglass control: the arithmetic of OpA with the sums
// split by whether their terms can cancel.  The corner differences (a_xi, a_eta of nearly equal
// nodal sums) and every node-level accumulation (corner combinations, carried and exchanged
// partials) use the accurate double-word addition; the contractions that form the strain, the
// stress and H = S M^-T, whose terms carry no such cancellation, use the fused multiply-add and the
// sum without the second TwoSum (add_nc / fma_nc).  The two wedges of the cell are the two lanes of
// packed f32x2 double-floats (x = W0, y = W1; lane pairs of corners (00, 11), (10, 01), (01, 10),
// as in OpA<float, false>), one issue slot per pair; lanes meet only where corners 10 and 01 and
// the top-minus-bottom parts combine.
template <>
struct OpA<dfl, false> {
  static constexpr int NIN = 3, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = true, NEEDS_D = true;
  struct Col {
    df2 M[9], dM;  // M^-1 entries and |det M| of (W0, W1)
  };
  int div_term;
  dfl hgk;
  __device__ __forceinline__ Col column(const dfl (&Mi)[2][9], const dfl (&dM)[2], int) const {
    Col c;
#pragma unroll
    for (int q = 0; q < 9; ++q) c.M[q] = pack(Mi[0][q], Mi[1][q]);
    c.dM = pack(dM[0], dM[1]);
    return c;
  }
  __device__ __forceinline__ void cell(const dfl (&s)[4][3], const dfl (&dd)[4][3], const dfl (&)[2][9],
                                       const dfl (&)[2], const dfl* lc, const dfl (&eta)[2], dfl (&accb)[4][3],
                                       dfl (&acct)[4][3], const Col& col) const {
    const df2 r = pack(lc[4], lc[4]), vw2 = pack(lc[5], lc[5]);
    const df2* M = col.M;
    const df2 mr[3] = {mul2(r, M[6]), mul2(r, M[7]), mul2(r, M[8])};
    df2 G[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const df2 s0 = pack(s[0][c], s[3][c]), s1 = pack(s[1][c], s[2][c]), s2 = pack(s[2][c], s[1][c]);
      const df2 ax = sub2(s1, s0), ay = sub2(s2, s0);
      const df2 az = add_nc2(add_nc2(pack(dd[0][c], dd[3][c]), pack(dd[1][c], dd[2][c])), pack(dd[2][c], dd[1][c]));
#pragma unroll
      for (int x = 0; x < 3; ++x) G[c][x] = fma_nc2(ax, M[x], fma_nc2(ay, M[3 + x], mul2(az, mr[x])));
    }
    const df2 ve = mul2(mul2(vw2, col.dM), pack(eta[0], eta[1]));
    const df2 ve2{p2add(ve.hi, ve.hi), p2add(ve.lo, ve.lo)};  // exact doubling
    df2 S[3][3];
    if (div_term) {
      const dfl m23(-2.0 / 3.0);
      const df2 vt = mul2(mul2(ve, pack(m23, m23)), add_nc2(add_nc2(G[0][0], G[1][1]), G[2][2]));
      S[0][0] = fma_nc2(ve2, G[0][0], vt), S[1][1] = fma_nc2(ve2, G[1][1], vt), S[2][2] = fma_nc2(ve2, G[2][2], vt);
    } else {
      S[0][0] = mul2(ve2, G[0][0]), S[1][1] = mul2(ve2, G[1][1]), S[2][2] = mul2(ve2, G[2][2]);
    }
    S[0][1] = S[1][0] = mul2(ve, add_nc2(G[0][1], G[1][0]));
    S[0][2] = S[2][0] = mul2(ve, add_nc2(G[0][2], G[2][0]));
    S[1][2] = S[2][1] = mul2(ve, add_nc2(G[1][2], G[2][1]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const df2 h0 = fma_nc2(S[c][0], M[0], fma_nc2(S[c][1], M[1], mul2(S[c][2], M[2])));
      const df2 h1 = fma_nc2(S[c][0], M[3], fma_nc2(S[c][1], M[4], mul2(S[c][2], M[5])));
      const df2 h2 = fma_nc2(S[c][0], mr[0], fma_nc2(S[c][1], mr[1], mul2(S[c][2], mr[2])));
      // X at corners (00, 11) = -(h0 + h1) per lane; at (10, 01) = (h0.x + h1.y, h1.x + h0.y)
      const df2 x03 = add2(h0, h1);
      const df2 x12 = add2(pack(lane_x(h0), lane_x(h1)), pack(lane_y(h1), lane_y(h0)));
      // top-minus-bottom part: h2 at (00, 11), h2.x + h2.y at (10, 01)
      const dfl hs = lane_x(h2) + lane_y(h2);
      const df2 h12 = pack(hs, hs);
      const df2 b03 = add2(x03, h2), t03 = sub2(h2, x03);  // bottom -(x03 + h2), top h2 - x03
      const df2 b12 = sub2(x12, h12), t12 = add2(x12, h12);
      accb[0][c] = -lane_x(b03), acct[0][c] = lane_x(t03);
      accb[3][c] = -lane_y(b03), acct[3][c] = lane_y(t03);
      accb[1][c] = lane_x(b12), acct[1][c] = lane_x(t12);
      accb[2][c] = lane_y(b12), acct[2][c] = lane_y(t12);
    }
  }
};

// Packed FP32 pairs (sm_100+ f32x2 instructions): one instruction per pair halves the issue
// slots of the FP32 element arithmetic, which bounds the FP32 tile kernels.
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b lane-wise, rounded to nearest: the packed subtraction of PTX (no intrinsic exists)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// FP32 viscous block without hourglass control: the same arithmetic as OpA with the two wedges
// of the cell as the two lanes of packed f32x2 values (x = W0, y = W1).  W0's corners (c0, c1,
// c2) are (00, 10, 01) and W1's are (11, 01, 10), so the lane pairs are (00, 11), (10, 01), (01, 10).
template <>
struct OpA<float, false> {
  static constexpr int NIN = 3, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = true, NEEDS_D = true;
  struct Col {
    float2 M[9], dM;  // M^-1 entries and |det M| of (W0, W1)
  };
  int div_term;
  float hgk;
  __device__ __forceinline__ Col column(const float (&Mi)[2][9], const float (&dM)[2], int) const {
    Col c;
#pragma unroll
    for (int q = 0; q < 9; ++q) c.M[q] = p2(Mi[0][q], Mi[1][q]);
    c.dM = p2(dM[0], dM[1]);
    return c;
  }
  __device__ __forceinline__ void cell(const float (&s)[4][3], const float (&dd)[4][3], const float (&)[2][9],
                                       const float (&)[2], const float* lc, const float (&eta)[2],
                                       float (&accb)[4][3], float (&acct)[4][3], const Col& col) const {
    const float2 r = p2(lc[4], lc[4]);
    const float2* M = col.M;
    const float2 mr[3] = {mul2(r, M[6]), mul2(r, M[7]), mul2(r, M[8])};
    float2 G[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 s0 = p2(s[0][c], s[3][c]), s1 = p2(s[1][c], s[2][c]), s2 = p2(s[2][c], s[1][c]);
      const float2 ax = sub2(s1, s0), ay = sub2(s2, s0);
      const float2 az = add2(add2(p2(dd[0][c], dd[3][c]), p2(dd[1][c], dd[2][c])), p2(dd[2][c], dd[1][c]));
#pragma unroll
      for (int x = 0; x < 3; ++x) G[c][x] = fma2(ax, M[x], fma2(ay, M[3 + x], mul2(az, mr[x])));
    }
    const float2 ve = mul2(mul2(p2(lc[5], lc[5]), col.dM), p2(eta[0], eta[1]));
    const float2 ve2 = add2(ve, ve);
    float2 S[3][3];
    if (div_term) {
      const float2 vt = mul2(mul2(ve, p2(-2.f / 3.f, -2.f / 3.f)), add2(add2(G[0][0], G[1][1]), G[2][2]));
      S[0][0] = fma2(ve2, G[0][0], vt), S[1][1] = fma2(ve2, G[1][1], vt), S[2][2] = fma2(ve2, G[2][2], vt);
    } else {
      S[0][0] = mul2(ve2, G[0][0]), S[1][1] = mul2(ve2, G[1][1]), S[2][2] = mul2(ve2, G[2][2]);
    }
    S[0][1] = S[1][0] = mul2(ve, add2(G[0][1], G[1][0]));
    S[0][2] = S[2][0] = mul2(ve, add2(G[0][2], G[2][0]));
    S[1][2] = S[2][1] = mul2(ve, add2(G[1][2], G[2][1]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 h0 = fma2(S[c][0], M[0], fma2(S[c][1], M[1], mul2(S[c][2], M[2])));
      const float2 h1 = fma2(S[c][0], M[3], fma2(S[c][1], M[4], mul2(S[c][2], M[5])));
      const float2 h2 = fma2(S[c][0], mr[0], fma2(S[c][1], mr[1], mul2(S[c][2], mr[2])));
      // X at corners (00, 11) = -(h0 + h1) per lane; at (10, 01) = (h0.x + h1.y, h1.x + h0.y)
      const float2 x03 = add2(h0, h1);
      const float2 x12 = add2(p2(h0.x, h1.x), p2(h1.y, h0.y));
      // top-minus-bottom part: h2 at (00, 11), h2.x + h2.y at (10, 01)
      const float hs = h2.x + h2.y;
      const float2 h12 = p2(hs, hs);
      const float2 b03 = add2(x03, h2), t03 = sub2(h2, x03);  // -(X) -/+ h2 negated: b = -(X - h2)
      const float2 b12 = sub2(x12, h12), t12 = add2(x12, h12);
      accb[0][c] = -b03.x, acct[0][c] = t03.x;
      accb[3][c] = -b03.y, acct[3][c] = t03.y;
      accb[1][c] = b12.x, acct[1][c] = t12.x;
      accb[2][c] = b12.y, acct[2][c] = t12.y;
    }
  }
};

// FP32 viscous block with hourglass control, packed as OpA<float, false>; the control follows
// the scalar OpA<T, true> (alpha_m, b_m, the H[:,0/1] corrections and the per-corner
// top-minus-bottom parts), lane x = W0, lane y = W1.
template <>
struct OpA<float, true> {
  static constexpr int NIN = 3, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = true, NEEDS_D = true;
  struct Col {
    float2 M[9], dM, eL, eR;
  };
  int div_term;
  float hgk;
  __device__ __forceinline__ Col column(const float (&Mi)[2][9], const float (&dM)[2], int) const {
    Col c;
#pragma unroll
    for (int q = 0; q < 9; ++q) c.M[q] = p2(Mi[0][q], Mi[1][q]);
    c.dM = p2(dM[0], dM[1]);
    const HgCol<float> h = hg_column(Mi, dM);
    c.eL = p2(h.eL[0], h.eL[1]), c.eR = p2(h.eR[0], h.eR[1]);
    return c;
  }
  __device__ __forceinline__ void cell(const float (&s)[4][3], const float (&dd)[4][3], const float (&)[2][9],
                                       const float (&)[2], const float* lc, const float (&eta)[2],
                                       float (&accb)[4][3], float (&acct)[4][3], const Col& col) const {
    const float2 r = p2(lc[4], lc[4]), k9 = p2(lc[8], lc[8]), nk9 = p2(-lc[8], -lc[8]);
    const float2 third = p2(1.f / 3.f, 1.f / 3.f);
    const float2* M = col.M;
    const float2 mr[3] = {mul2(r, M[6]), mul2(r, M[7]), mul2(r, M[8])};
    float2 G[3][3], al1[3], al2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 s0 = p2(s[0][c], s[3][c]), s1 = p2(s[1][c], s[2][c]), s2 = p2(s[2][c], s[1][c]);
      const float2 d1 = p2(dd[1][c], dd[2][c]), d2 = p2(dd[2][c], dd[1][c]);
      const float2 ax = sub2(s1, s0), ay = sub2(s2, s0);
      const float2 az = add2(add2(p2(dd[0][c], dd[3][c]), d1), d2);
#pragma unroll
      for (int x = 0; x < 3; ++x) G[c][x] = fma2(ax, M[x], fma2(ay, M[3 + x], mul2(az, mr[x])));
      const float2 a3 = mul2(az, third);
      al1[c] = fma2(nk9, sub2(add2(ax, ax), ay), sub2(d1, a3));
      al2[c] = fma2(nk9, sub2(add2(ay, ay), ax), sub2(d2, a3));
    }
    const float2 ve = mul2(mul2(p2(lc[5], lc[5]), col.dM), p2(eta[0], eta[1]));
    const float2 ve2 = add2(ve, ve);
    float2 S[3][3];
    if (div_term) {
      const float2 vt = mul2(mul2(ve, p2(-2.f / 3.f, -2.f / 3.f)), add2(add2(G[0][0], G[1][1]), G[2][2]));
      S[0][0] = fma2(ve2, G[0][0], vt), S[1][1] = fma2(ve2, G[1][1], vt), S[2][2] = fma2(ve2, G[2][2], vt);
    } else {
      S[0][0] = mul2(ve2, G[0][0]), S[1][1] = mul2(ve2, G[1][1]), S[2][2] = mul2(ve2, G[2][2]);
    }
    S[0][1] = S[1][0] = mul2(ve, add2(G[0][1], G[1][0]));
    S[0][2] = S[2][0] = mul2(ve, add2(G[0][2], G[2][0]));
    S[1][2] = S[2][1] = mul2(ve, add2(G[1][2], G[2][1]));
    const float2 eps = mul2(mul2(p2(hgk, hgk), p2(eta[0], eta[1])),
                            fma2(p2(lc[5], lc[5]), col.eL, mul2(p2(lc[9], lc[9]), col.eR)));
    const float2 nek = mul2(eps, nk9), e3 = mul2(eps, third);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 b1 = sub2(add2(al1[c], al1[c]), al2[c]), b2 = sub2(add2(al2[c], al2[c]), al1[c]);
      const float2 h0 = fma2(nek, b1, fma2(S[c][0], M[0], fma2(S[c][1], M[1], mul2(S[c][2], M[2]))));
      const float2 h1 = fma2(nek, b2, fma2(S[c][0], M[3], fma2(S[c][1], M[4], mul2(S[c][2], M[5]))));
      const float2 h2 = fma2(S[c][0], mr[0], fma2(S[c][1], mr[1], mul2(S[c][2], mr[2])));
      const float2 v1 = mul2(e3, b1), v2 = mul2(e3, b2);
      const float2 y0 = sub2(h2, add2(v1, v2)), y1 = add2(h2, v1), y2 = add2(h2, v2);
      // X: (00, 11) = -(h0 + h1); (10, 01) = (h0.x + h1.y, h1.x + h0.y).  Y: (00, 11) = y0;
      // (10, 01) = (y1.x + y2.y, y2.x + y1.y).
      const float2 x03 = add2(h0, h1);
      const float2 x12 = add2(p2(h0.x, h1.x), p2(h1.y, h0.y));
      const float2 y12 = add2(p2(y1.x, y2.x), p2(y2.y, y1.y));
      const float2 b03 = add2(x03, y0), t03 = sub2(y0, x03);
      const float2 b12 = sub2(x12, y12), t12 = add2(x12, y12);
      accb[0][c] = -b03.x, acct[0][c] = t03.x;
      accb[3][c] = -b03.y, acct[3][c] = t03.y;
      accb[1][c] = b12.x, acct[1][c] = t12.x;
      accb[2][c] = b12.y, acct[2][c] = t12.y;
    }
  }
};

// Viscous block with a second radial quadrature point: the two-point Gauss rule in zeta at the
// lateral barycentre, zeta = -/+ z (z = 1/sqrt 3), weight 1/2 each, one eta per wedge.  At
// zeta the scaled strain is G0 + zeta G1: G0 is the one-point G' above and
// G1 = b_xi M^-1[0,:] + b_eta M^-1[1,:] + (a_zeta / 3) M^-1[2,:], b_xi = d_c1 - d_c0,
// b_eta = d_c2 - d_c0 (the lateral gradient of the radial differences; r_q = r + zeta / 3), and
// V_q w0_q^2 = vol w0^2 / 2 at both points.  Summed over the two points, with S0 the stress of
// G0 (factor vol w0^2 |det M| eta) and S1' that of G1 with a third of that factor, node
// (a, bottom / top) receives X_a -/+ D_a: X = (-S0 m0 - S0 m1, S0 m0, S0 m1) as in OpA and
// D_a = (-(S1' m0 + S1' m1), S1' m0, S1' m1)_a + S0 r m2 + S1' m2 / 3.
template <typename T>
struct OpA2 {
  static constexpr int NIN = 3, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = true, NEEDS_D = true;
  using Col = NoCol;
  int div_term;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int) const { return Col{}; }
  __device__ __forceinline__ static void stress(const T (&G)[3][3], T f, int div_term, T (&S)[3][3]) {
    const T f2 = f + f;
    if (div_term) {
      const T vt = (f * (T)(-2.0 / 3.0)) * ((G[0][0] + G[1][1]) + G[2][2]);
      S[0][0] = f2 * G[0][0] + vt, S[1][1] = f2 * G[1][1] + vt, S[2][2] = f2 * G[2][2] + vt;
    } else {
      S[0][0] = f2 * G[0][0], S[1][1] = f2 * G[1][1], S[2][2] = f2 * G[2][2];
    }
    S[0][1] = S[1][0] = f * (G[0][1] + G[1][0]);
    S[0][2] = S[2][0] = f * (G[0][2] + G[2][0]);
    S[1][2] = S[2][1] = f * (G[1][2] + G[2][1]);
  }
  __device__ __forceinline__ void cell(const T (&s)[4][3], const T (&dd)[4][3], const T (&Mi)[2][9],
                                       const T (&dM)[2], const T* lc, const T (&eta)[2], T (&accb)[4][3],
                                       T (&acct)[4][3], const Col&) const {
    const T r = lc[4], vw2 = lc[5];
    T X[4][3], Y[4][3];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int c0 = kCorner[w][0], c1 = kCorner[w][1], c2 = kCorner[w][2];
      const T* M = Mi[w];
      const T mr[3] = {r * M[6], r * M[7], r * M[8]};
      const T m3[3] = {M[6] * (T)(1.0 / 3.0), M[7] * (T)(1.0 / 3.0), M[8] * (T)(1.0 / 3.0)};
      T S0[3][3], S1[3][3];
      {
        T G0[3][3], G1[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T ax = s[c1][c] - s[c0][c], ay = s[c2][c] - s[c0][c], az = (dd[c0][c] + dd[c1][c]) + dd[c2][c];
          const T bx = dd[c1][c] - dd[c0][c], by = dd[c2][c] - dd[c0][c];
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            G0[c][x] = ax * M[x] + ay * M[3 + x] + az * mr[x];
            G1[c][x] = bx * M[x] + by * M[3 + x] + az * m3[x];
          }
        }
        const T ve = vw2 * dM[w] * eta[w];
        stress(G0, ve, div_term, S0);
        stress(G1, ve * (T)(1.0 / 3.0), div_term, S1);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T h0 = S0[c][0] * M[0] + S0[c][1] * M[1] + S0[c][2] * M[2];
        const T h1 = S0[c][0] * M[3] + S0[c][1] * M[4] + S0[c][2] * M[5];
        const T k0 = S1[c][0] * M[0] + S1[c][1] * M[1] + S1[c][2] * M[2];
        const T k1 = S1[c][0] * M[3] + S1[c][1] * M[4] + S1[c][2] * M[5];
        const T hc = (S0[c][0] * mr[0] + S0[c][1] * mr[1] + S0[c][2] * mr[2]) +
                     (S1[c][0] * m3[0] + S1[c][1] * m3[1] + S1[c][2] * m3[2]);
        Y[c0][c] = hc - (k0 + k1);
        X[c0][c] = -(h0 + h1);
        if (w == 0) {
          Y[c1][c] = hc + k0, Y[c2][c] = hc + k1;
          X[c1][c] = h0, X[c2][c] = h1;
        } else {
          Y[c1][c] += hc + k0, Y[c2][c] += hc + k1;
          X[c1][c] += h0, X[c2][c] += h1;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) accb[q][c] = X[q][c] - Y[q][c], acct[q][c] = X[q][c] + Y[q][c];
  }
};

// Fine-level divergence: each of the six nodes of a wedge gets -V tr(grad u)(q_c) / 6
// (pressure test function psi = N_n with N_n(q_c) = 1/6); tr grad u = w0 tr G'.
// RHO (TALA, Eq. mass): -V (rho(q_c) div u_h(q_c) + rho'(q_c) r_hat(q_c) . u_h(q_c)) / 6, the
// product rule at the quadrature point; the layer table carries rho(q_c) in slot 10 and
// rho'(q_c) / (6 w0) in slot 11, u_h(q_c) is the sum of the wedge's three corner sums (top + bottom)
// over 6, so the bracket is w0 (slot 10 tr G' + slot 11 r_hat . sum_a s_a); r_hat(q_c) per lateral
// triangle comes from the level's table.
template <typename T, bool RHO = false>
struct OpDiv {
  static constexpr int NIN = 3, NOUT = 1;
  static constexpr bool USES_ETA = false, LOADS = true, NEEDS_D = true;
  struct ColR {
    T rh[2][3];
  };
  using Col = typename std::conditional<RHO, ColR, NoCol>::type;
  const T* rhat = nullptr;  // [3][n_tri] r_hat(q_c) of every lateral triangle (RHO only)
  int n_tri = 0;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int t0) const {
    if constexpr (RHO) {
      ColR c;
#pragma unroll
      for (int w = 0; w < 2; ++w)
#pragma unroll
        for (int x = 0; x < 3; ++x) c.rh[w][x] = rhat[x * n_tri + t0 + w];
      return c;
    } else {
      return Col{};
    }
  }
  __device__ __forceinline__ void cell(const T (&s)[4][3], const T (&dd)[4][3], const T (&Mi)[2][9],
                                       const T (&dM)[2], const T* lc, const T (&)[2], T (&accb)[4][1],
                                       T (&acct)[4][1], const Col& col) const {
    const T r = lc[4], vw6 = lc[7];
    T v[2];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int c0 = kCorner[w][0], c1 = kCorner[w][1], c2 = kCorner[w][2];
      const T* M = Mi[w];
      T lat = 0, rad = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T ax = s[c1][c] - s[c0][c], ay = s[c2][c] - s[c0][c], az = (dd[c0][c] + dd[c1][c]) + dd[c2][c];
        lat = c == 0 ? ax * M[0] + ay * M[3] : lat + ax * M[c] + ay * M[3 + c];
        rad = c == 0 ? az * M[6] : rad + az * M[6 + c];
      }
      T div = lat + r * rad;
      if constexpr (RHO) {
        T rs = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T sc = (s[c0][c] + s[c1][c]) + s[c2][c];
          rs = c == 0 ? col.rh[w][0] * sc : rs + col.rh[w][c] * sc;
        }
        div = lc[10] * div + lc[11] * rs;
      }
      v[w] = (vw6 * dM[w]) * div;
    }
    const T v01 = v[0] + v[1];
    accb[0][0] = acct[0][0] = v[0];
    accb[3][0] = acct[3][0] = v[1];
    accb[1][0] = acct[1][0] = v01;
    accb[2][0] = acct[2][0] = v01;
  }
};

// Double-float divergence without the TALA term: the arithmetic of OpDiv with the corner
// differences and the corner combination of the two wedges accurate, the contraction with M^-1 by
// fused multiply-adds (add_nc / fma_nc), the two wedges in the lanes of packed double-floats.
template <>
struct OpDiv<dfl, false> {
  static constexpr int NIN = 3, NOUT = 1;
  static constexpr bool USES_ETA = false, LOADS = true, NEEDS_D = true, PREFETCH = true;
  struct Col {
    df2 M[9], dM;  // M^-1 entries and |det M| of (W0, W1)
  };
  const dfl* rhat = nullptr;
  int n_tri = 0;
  __device__ __forceinline__ Col column(const dfl (&Mi)[2][9], const dfl (&dM)[2], int) const {
    Col c;
#pragma unroll
    for (int q = 0; q < 9; ++q) c.M[q] = pack(Mi[0][q], Mi[1][q]);
    c.dM = pack(dM[0], dM[1]);
    return c;
  }
  // the two wedges in the lanes of packed double-floats (x = W0, y = W1), corner pairs as in
  // OpA<dfl, false>: a_xi = s_10 - s_00 | s_01 - s_11, a_eta = s_01 - s_00 | s_10 - s_11
  __device__ __forceinline__ void cell(const dfl (&s)[4][3], const dfl (&dd)[4][3], const dfl (&)[2][9],
                                       const dfl (&)[2], const dfl* lc, const dfl (&)[2], dfl (&accb)[4][1],
                                       dfl (&acct)[4][1], const Col& col) const {
    const df2 r = pack(lc[4], lc[4]), vw6 = pack(lc[7], lc[7]);
    const df2* M = col.M;
    df2 lat, rad;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const df2 s0 = pack(s[0][c], s[3][c]), s1 = pack(s[1][c], s[2][c]), s2 = pack(s[2][c], s[1][c]);
      const df2 ax = sub2(s1, s0), ay = sub2(s2, s0);
      const dfl d12 = add_nc(dd[1][c], dd[2][c]);
      const df2 az = add_nc2(pack(dd[0][c], dd[3][c]), pack(d12, d12));
      lat = c == 0 ? fma_nc2(ax, M[0], mul2(ay, M[3])) : fma_nc2(ax, M[c], fma_nc2(ay, M[3 + c], lat));
      rad = c == 0 ? mul2(az, M[6]) : fma_nc2(az, M[6 + c], rad);
    }
    const df2 v = mul2(mul2(vw6, col.dM), fma_nc2(r, rad, lat));
    const dfl v01 = lane_x(v) + lane_y(v);
    accb[0][0] = acct[0][0] = lane_x(v);
    accb[3][0] = acct[3][0] = lane_y(v);
    accb[1][0] = acct[1][0] = v01;
    accb[2][0] = acct[2][0] = v01;
  }
};

// Fine-level gradient (transpose of OpDiv): y_j += -V p(q_c) grad N_j(q_c), p(q_c) the mean of
// the six nodal values; H[:, m] = f M^-1[m, :] (times r for m = 2), f = -vol w0 |det M| p(q_c).
template <typename T>
struct OpGrad {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = false, LOADS = true, NEEDS_D = false;
  using Col = NoCol;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int) const { return Col{}; }
  __device__ __forceinline__ void cell(const T (&sn)[4][1], const T (&)[4][1], const T (&Mi)[2][9],
                                       const T (&dM)[2], const T* lc, const T (&)[2], T (&accb)[4][3],
                                       T (&acct)[4][3], const Col&) const {
    const T r = lc[4], vw6 = lc[7];
    const T s[4] = {sn[0][0], sn[1][0], sn[2][0], sn[3][0]};
    T X[4][3], h[2][3];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int c0 = kCorner[w][0], c1 = kCorner[w][1], c2 = kCorner[w][2];
      const T* M = Mi[w];
      const T f = (vw6 * dM[w]) * ((s[c0] + s[c1]) + s[c2]);
      const T fr = f * r;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T h0 = f * M[c], h1 = f * M[3 + c];
        h[w][c] = fr * M[6 + c];
        X[c0][c] = -(h0 + h1);
        if (w == 0) {
          X[c1][c] = h0, X[c2][c] = h1;
        } else {
          X[c1][c] += h0, X[c2][c] += h1;
        }
      }
    }
    combine_corners<T, 3>(X, h, accb, acct);
  }
};

// Double-float gradient: the pressure sum at q_c (no cancellation) and the products by M^-1 with the
// sum without the second TwoSum; the corner combination accurate; the two wedges in the lanes of
// packed double-floats.
template <>
struct OpGrad<dfl> {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = false, LOADS = true, NEEDS_D = false, PREFETCH = true;
  struct Col {
    df2 M[9], dM;  // M^-1 entries and |det M| of (W0, W1)
  };
  __device__ __forceinline__ Col column(const dfl (&Mi)[2][9], const dfl (&dM)[2], int) const {
    Col c;
#pragma unroll
    for (int q = 0; q < 9; ++q) c.M[q] = pack(Mi[0][q], Mi[1][q]);
    c.dM = pack(dM[0], dM[1]);
    return c;
  }
  // the two wedges in the lanes of packed double-floats (x = W0, y = W1); corners as in OpA<dfl, false>
  __device__ __forceinline__ void cell(const dfl (&sn)[4][1], const dfl (&)[4][1], const dfl (&)[2][9],
                                       const dfl (&)[2], const dfl* lc, const dfl (&)[2], dfl (&accb)[4][3],
                                       dfl (&acct)[4][3], const Col& col) const {
    const df2 r = pack(lc[4], lc[4]), vw6 = pack(lc[7], lc[7]);
    const df2* M = col.M;
    const dfl s12 = add_nc(sn[1][0], sn[2][0]);  // corners 10 and 01 belong to both wedges
    const df2 f = mul2(mul2(vw6, col.dM), add_nc2(pack(sn[0][0], sn[3][0]), pack(s12, s12)));
    const df2 fr = mul2(f, r);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const df2 h0 = mul2(f, M[c]), h1 = mul2(f, M[3 + c]), h2 = mul2(fr, M[6 + c]);
      const df2 x03 = add2(h0, h1);
      const df2 x12 = add2(pack(lane_x(h0), lane_x(h1)), pack(lane_y(h1), lane_y(h0)));
      const dfl hs = lane_x(h2) + lane_y(h2);
      const df2 h12 = pack(hs, hs);
      const df2 b03 = add2(x03, h2), t03 = sub2(h2, x03);  // bottom -(x03 + h2), top h2 - x03
      const df2 b12 = sub2(x12, h12), t12 = add2(x12, h12);
      accb[0][c] = -lane_x(b03), acct[0][c] = lane_x(t03);
      accb[3][c] = -lane_y(b03), acct[3][c] = lane_y(t03);
      accb[1][c] = lane_x(b12), acct[1][c] = lane_x(t12);
      accb[2][c] = lane_y(b12), acct[2][c] = lane_y(t12);
    }
  }
};

// Diagonal of A (no input): node j of a wedge receives V eta (|g_j|^2 + c g_j[d]^2) for each
// component d, g_j = grad N_j(q_c) = w0 (l_a -/+ r m2) (bottom / top), with m_k the rows of M^-1,
// l_0 = -(m0 + m1), l_1 = m0, l_2 = m1, r = w1 / w0, and c = 1/3 with the -2/3 div term, 1 without
// (A_jj = V eta (|g|^2 I + c g g^T)).  Expanded:
//   V eta w0^2 (P_ad + r^2 Q_d -/+ 2 r R_ad),
//   P_ad = |l_a|^2 + c l_ad^2, Q_d = |m2|^2 + c m2_d^2, R_ad = l_a . m2 + c l_ad m2_d,
// whose 21 factors depend on the lateral triangle only: they come from a per-level table
// (Level::dcoef64 / dcoef32), so a cell costs three FMAs per node and component.  V eta w0^2 = vol w0^2 |det M|
// eta.  With HG, node (a, side) also gets eps (g_1,j^2 + g_2,j^2) in every component, which is
// eps n_a (k9 - zeta / 3)^2 with n_a = 2, 5, 5 for a = 0, 1, 2 (zeta = -1 bottom, +1 top).

template <typename T, bool HG = false>
struct OpDiag {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = false, NEEDS_D = false;
  struct Col {
    int t0;
  };
  int div_term;
  T hgk;
  const T* coef;  // [kDiagCoef][n_tri]
  int n_tri;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int t0) const { return Col{t0}; }
  __device__ __forceinline__ void cell(const T (&)[4][1], const T (&)[4][1], const T (&)[2][9], const T (&dM)[2],
                                       const T* lc, const T (&eta)[2], T (&accb)[4][3], T (&acct)[4][3],
                                       const Col& col) const {
    const T r = lc[4], vw2 = lc[5];
    const T r2 = r * r, rr = r + r;
    T kbb = 0, ktt = 0;
    if constexpr (HG) {
      const T kb = lc[8] + (T)(1.0 / 3.0), kt = lc[8] - (T)(1.0 / 3.0);
      kbb = kb * kb, ktt = kt * kt;
    }
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const T* cf = coef + col.t0 + w;
      const T A = vw2 * dM[w] * eta[w];
      const T Ar2 = A * r2, A2r = A * rr;
      T hb = 0, ht = 0;
      if constexpr (HG) {
        const T eps = (hgk * eta[w]) * dM[w] * (vw2 * cf[21 * n_tri] + lc[9] * cf[22 * n_tri]);
        hb = eps * kbb, ht = eps * ktt;
      }
      T AQ[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) AQ[d] = Ar2 * cf[(18 + d) * n_tri];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = kCorner[w][a];
        const bool first = w == 0 || q == 3;  // corner 11 belongs to W1 only
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T inner = A * cf[(3 * a + d) * n_tri] + AQ[d];
          const T cr = A2r * cf[(9 + 3 * a + d) * n_tri];
          T vb = inner - cr, vt = inner + cr;
          if constexpr (HG) {
            const T na = a == 0 ? (T)2 : (T)5;
            vb += na * hb, vt += na * ht;
          }
          accb[q][d] = first ? vb : accb[q][d] + vb;
          acct[q][d] = first ? vt : acct[q][d] + vt;
        }
      }
    }
  }
};

// Energy residual of Eq. (energy) in the nondimensional Boussinesq form, dT/dt + u . grad T = lap T,
// one-point rule (inputs u_x, u_y, u_z, T; one output): node j of a wedge receives
//   grad N_j . F + V a / 6,   F = V (grad T + tau a ubar),   a = ubar . grad T,
// the diffusion, the Galerkin advection (N_j(q_c) = 1/6) and, with supg, the streamline-upwind term
// of SUPG (Brooks and Hughes 1982); all at q_c, ubar the mean of the six nodal velocities,
// tau = h / (2 |ubar|) (coth Pe - 1 / Pe), Pe = |ubar| h / 2, h = (2 V)^(1/3) (the hexahedral cell's
// volume), with the series h^2 / 12 (1 - Pe^2 / 15) for Pe < 1e-3.  grad T = w0 G with G formed from
// the corner sums / differences as the strain of OpA, grad N_j = w0 (l_a -/+ r m2) (bottom / top).
// adv = 0: diffusion only (the inputs' velocity slots are not used).
template <typename T>
struct OpEnergy {
  static constexpr int NIN = 4, NOUT = 1;
  static constexpr bool USES_ETA = false, LOADS = true, NEEDS_D = true;
  using Col = NoCol;
  int adv, supg;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int) const { return Col{}; }
  __device__ __forceinline__ void cell(const T (&s)[4][4], const T (&dd)[4][4], const T (&Mi)[2][9],
                                       const T (&dM)[2], const T* lc, const T (&)[2], T (&accb)[4][1],
                                       T (&acct)[4][1], const Col&) const {
    const T w0 = lc[0], vol = lc[2], r = lc[4];
    T yb[2][3], yt[2][3];
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int c0 = kCorner[w][0], c1 = kCorner[w][1], c2 = kCorner[w][2];
      const T* M = Mi[w];
      const T ax = s[c1][3] - s[c0][3], ay = s[c2][3] - s[c0][3], az = (dd[c0][3] + dd[c1][3]) + dd[c2][3];
      T G[3], F[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) G[x] = ax * M[x] + ay * M[3 + x] + az * (r * M[6 + x]);
      const T V = vol * dM[w];
#pragma unroll
      for (int x = 0; x < 3; ++x) F[x] = (V * w0) * G[x];
      T q = 0;
      if (adv) {
        T ub[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) ub[x] = ((s[c0][x] + s[c1][x]) + s[c2][x]) * (T)(1.0 / 6.0);
        const T a = w0 * ((ub[0] * G[0] + ub[1] * G[1]) + ub[2] * G[2]);
        q = V * a * (T)(1.0 / 6.0);
        if (supg) {
          const T un = sqrt((ub[0] * ub[0] + ub[1] * ub[1]) + ub[2] * ub[2]);
          const T h = cbrt((T)2 * V);
          const T pe = un * h * (T)0.5;
          const T tau = pe > (T)1e-3 ? h / ((T)2 * un) * ((T)1 / tanh(pe) - (T)1 / pe)
                                     : h * h * (T)(1.0 / 12.0) * ((T)1 - pe * pe * (T)(1.0 / 15.0));
          const T ta = V * tau * a;
#pragma unroll
          for (int x = 0; x < 3; ++x) F[x] += ta * ub[x];
        }
      }
      const T p0 = (M[0] * F[0] + M[1] * F[1]) + M[2] * F[2];
      const T p1 = (M[3] * F[0] + M[4] * F[1]) + M[5] * F[2];
      const T p2 = r * ((M[6] * F[0] + M[7] * F[1]) + M[8] * F[2]);
      const T lat[3] = {-(p0 + p1), p0, p1};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        yb[w][a] = w0 * (lat[a] - p2) + q;
        yt[w][a] = w0 * (lat[a] + p2) + q;
      }
    }
    // corners: 00 <- W0 node 0; 11 <- W1 node 0; 10 <- W0 node 1 + W1 node 2; 01 <- W0 node 2 + W1 node 1
    accb[0][0] = yb[0][0], acct[0][0] = yt[0][0];
    accb[3][0] = yb[1][0], acct[3][0] = yt[1][0];
    accb[1][0] = yb[0][1] + yb[1][2], acct[1][0] = yt[0][1] + yt[1][2];
    accb[2][0] = yb[0][2] + yb[1][1], acct[2][0] = yt[0][2] + yt[1][1];
  }
};

// Lumped mass m_j = sum_e V_e / 6 (no input).
template <typename T>
struct OpMass {
  static constexpr int NIN = 1, NOUT = 1;
  static constexpr bool USES_ETA = false, LOADS = false, NEEDS_D = false;
  using Col = NoCol;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int) const { return Col{}; }
  __device__ __forceinline__ void cell(const T (&)[4][1], const T (&)[4][1], const T (&)[2][9], const T (&dM)[2],
                                       const T* lc, const T (&)[2], T (&accb)[4][1], T (&acct)[4][1],
                                       const Col&) const {
    const T v0 = lc[2] * dM[0] * (T)(1.0 / 6.0), v1 = lc[2] * dM[1] * (T)(1.0 / 6.0);
    const T v01 = v0 + v1;
    accb[0][0] = acct[0][0] = v0;
    accb[3][0] = acct[3][0] = v1;
    accb[1][0] = acct[1][0] = v01;
    accb[2][0] = acct[2][0] = v01;
  }
};

// Double-float diagonal (one-point, no hourglass control): sums of positive terms, so every
// addition but the accumulation over the two wedges uses add_nc / fma_nc.
// Double-float diagonal without hourglass control, the two wedges of the cell in the lanes of
// packed df2 values (x = W0, y = W1) as in OpA<dfl, false>; the factor table comes per cell
// (Level::dcoefdf2), one 16-byte load per factor for both wedges.  Every contribution is a sum of
// squares, so the node sums of the tile kernel (POSITIVE) and the corner sums here use the
// double-word addition without the second TwoSum, which is accurate for operands of one sign.
template <>
struct OpDiag<dfl, false> {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = false, NEEDS_D = false, POSITIVE = true;
  struct Col {
    int p0;  // the cell's entry of the per-cell table
  };
  int div_term;
  dfl hgk;
  const float4* coef;  // [kDiagCoef][n_tri / 2]
  int n_pair;
  __device__ __forceinline__ Col column(const dfl (&)[2][9], const dfl (&)[2], int t0) const { return Col{t0 >> 1}; }
  __device__ __forceinline__ void cell(const dfl (&)[4][1], const dfl (&)[4][1], const dfl (&)[2][9], const dfl (&dM)[2],
                                       const dfl* lc, const dfl (&eta)[2], dfl (&accb)[4][3], dfl (&acct)[4][3],
                                       const Col& col) const {
    const df2 r = pack(lc[4], lc[4]), vw2 = pack(lc[5], lc[5]);
    const df2 r2 = mul2(r, r), rr{p2add(r.hi, r.hi), p2add(r.lo, r.lo)};  // exact doubling
    const df2 A = mul2(mul2(vw2, pack(dM[0], dM[1])), pack(eta[0], eta[1]));
    const df2 Ar2 = mul2(A, r2), A2r = mul2(A, rr);
    const float4* const cf = coef + col.p0;
    auto C = [&](int q) {
      const float4 v = cf[(int64_t)q * n_pair];
      return df2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
    };
    df2 AQ[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) AQ[d] = mul2(Ar2, C(18 + d));
    df2 vb[3][3], vt[3][3];  // local node a, component d; lanes (W0, W1)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const df2 inner = fma_nc2(A, C(3 * a + d), AQ[d]);
        const df2 cr = mul2(A2r, C(9 + 3 * a + d));
        vb[a][d] = add_nc2(inner, df2{p2neg(cr.hi), p2neg(cr.lo)});
        vt[a][d] = add_nc2(inner, cr);
      }
    // corners: 00 = W0 node 0, 11 = W1 node 0, 10 = W0 node 1 + W1 node 2, 01 = W0 node 2 + W1 node 1
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      accb[0][d] = lane_x(vb[0][d]), acct[0][d] = lane_x(vt[0][d]);
      accb[3][d] = lane_y(vb[0][d]), acct[3][d] = lane_y(vt[0][d]);
      const df2 b12 = add_nc2(pack(lane_x(vb[1][d]), lane_x(vb[2][d])), pack(lane_y(vb[2][d]), lane_y(vb[1][d])));
      const df2 t12 = add_nc2(pack(lane_x(vt[1][d]), lane_x(vt[2][d])), pack(lane_y(vt[2][d]), lane_y(vt[1][d])));
      accb[1][d] = lane_x(b12), accb[2][d] = lane_y(b12);
      acct[1][d] = lane_x(t12), acct[2][d] = lane_y(t12);
    }
  }
};

// Diagonal in gradient form (the FP32 path, where the table loads cost more than the arithmetic
// they save): node (a, side) of a wedge gets ve (|g|^2 + c g_d^2) with g = l_a w0 -/+ w1 m2
// formed per cell, plus the hourglass term of OpDiag.
template <typename T, bool HG = false>
struct OpDiagG {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = false, NEEDS_D = false;
  using Col = typename std::conditional<HG, HgCol<T>, NoCol>::type;
  int div_term;
  T hgk;
  __device__ __forceinline__ Col column(const T (&Mi)[2][9], const T (&dM)[2], int) const {
    if constexpr (HG) return hg_column(Mi, dM);
    else return Col{};
  }
  __device__ __forceinline__ void cell(const T (&)[4][1], const T (&)[4][1], const T (&Mi)[2][9], const T (&dM)[2],
                                       const T* lc, const T (&eta)[2], T (&accb)[4][3], T (&acct)[4][3],
                                       const Col& col) const {
    const T w0 = lc[0], w1 = lc[1], vol = lc[2];
    const T third = div_term ? (T)(1.0 / 3.0) : (T)1;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) accb[q][c] = acct[q][c] = 0;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const T* M = Mi[w];
      const T ve = vol * dM[w] * eta[w];
      T hb = 0, ht = 0;  // eps (k9 + 1/3)^2 and eps (k9 - 1/3)^2
      if constexpr (HG) {
        const T eps = (hgk * eta[w]) * (lc[5] * col.eL[w] + lc[9] * col.eR[w]);
        const T kb = lc[8] + (T)(1.0 / 3.0), kt = lc[8] - (T)(1.0 / 3.0);
        hb = eps * (kb * kb), ht = eps * (kt * kt);
      }
      T lat[3][3], u2[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const T u0 = w0 * M[x], u1 = w0 * M[3 + x];
        u2[x] = w1 * M[6 + x];
        lat[0][x] = -(u0 + u1), lat[1][x] = u0, lat[2][x] = u1;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = kCorner[w][a];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          T g[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) g[x] = side == 0 ? lat[a][x] - u2[x] : lat[a][x] + u2[x];
          const T g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          T hs = 0;
          if constexpr (HG) hs = (a == 0 ? (T)2 : (T)5) * (side == 0 ? hb : ht);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            T v = ve * (g2 + third * (g[c] * g[c]));
            if constexpr (HG) v += hs;
            if (side == 0) accb[q][c] += v;
            else acct[q][c] += v;
          }
        }
      }
    }
  }
};

// Diagonal with the second radial quadrature point (see OpA2): node (a, side) of a wedge gets
// ve (|g0|^2 + c g0_d^2) + ve / 3 (|g1|^2 + c g1_d^2), ve = vol w0^2 |det M| eta, with the
// one-point gradient g0 = l_a -/+ r m2 and g1 = l_a + m2 / 3 (the same on both sides), l_a the
// lateral gradient (-(m0 + m1), m0, m1)_a: the two points' gradients are g0 +/- z g1 (signed by
// side), whose squares sum to 2 (|g0|^2 + |g1|^2 / 3) times the weight 1/2.
template <typename T>
struct OpDiag2 {
  static constexpr int NIN = 1, NOUT = 3;
  static constexpr bool USES_ETA = true, LOADS = false, NEEDS_D = false;
  using Col = NoCol;
  int div_term;
  __device__ __forceinline__ Col column(const T (&)[2][9], const T (&)[2], int) const { return Col{}; }
  __device__ __forceinline__ void cell(const T (&)[4][1], const T (&)[4][1], const T (&Mi)[2][9], const T (&dM)[2],
                                       const T* lc, const T (&eta)[2], T (&accb)[4][3], T (&acct)[4][3],
                                       const Col&) const {
    const T r = lc[4], vw2 = lc[5];
    const T third = div_term ? (T)(1.0 / 3.0) : (T)1;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) accb[q][c] = acct[q][c] = 0;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const T* M = Mi[w];
      const T ve = vw2 * dM[w] * eta[w], ve3 = ve * (T)(1.0 / 3.0);
      T lat[3][3], mr[3], m3[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        lat[0][x] = -(M[x] + M[3 + x]), lat[1][x] = M[x], lat[2][x] = M[3 + x];
        mr[x] = r * M[6 + x], m3[x] = M[6 + x] * (T)(1.0 / 3.0);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = kCorner[w][a];
        T g1[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) g1[x] = lat[a][x] + m3[x];
        const T n1 = g1[0] * g1[0] + g1[1] * g1[1] + g1[2] * g1[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          T g[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) g[x] = side == 0 ? lat[a][x] - mr[x] : lat[a][x] + mr[x];
          const T n0 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T v = ve * (n0 + third * (g[c] * g[c])) + ve3 * (n1 + third * (g1[c] * g1[c]));
            if (side == 0) accb[q][c] += v;
            else acct[q][c] += v;
          }
        }
      }
    }
  }
};

// ------------------------------------------------------------------------------------ tile kernel
// Boundary handling flags of the tile kernel.
enum { PROJ_IN = 1, PROJ_OUT = 2, ADD_ID = 4 };

template <typename T>
__device__ __forceinline__ void project_vec(T (&v)[3], const T* s, int64_t soff, int64_t sstride, int bc) {
  if (bc == TN_BC_NOSLIP) {
    v[0] = v[1] = v[2] = (T)0;
    return;
  }
  T sx = s[soff], sy = s[soff + sstride], sz = s[soff + 2 * sstride];
  T dot = v[0] * sx + v[1] * sy + v[2] * sz;
  v[0] -= dot * sx, v[1] -= dot * sy, v[2] -= dot * sz;
}

// L1 prefetch of one global address (no register result).
template <typename T>
__device__ __forceinline__ void prefetch_l1(const T* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Fused vector update at node idx from y = (K x)(idx) (see EpiArgs); `in` is the apply input.
template <typename T, int EPI>
__device__ __forceinline__ void epilogue(const EpiArgs<T>& E, const T* in0, const T* in1, const T* in2, int idx,
                                         const T (&y)[3]) {
  if (EPI == EPI_RESID) {
#pragma unroll
    for (int c = 0; c < 3; ++c) E.r[c][idx] = E.b[c][idx] - y[c];
    return;
  }
  T rr[3];
  if (EPI == EPI_CHEB1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) rr[c] = E.b[c][idx] - y[c];
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) rr[c] = E.r[c][idx] - y[c];
  }
  const T a = E.binv[0][idx], e = E.binv[1][idx], f = E.binv[2][idx], xy = E.binv[3][idx], xz = E.binv[4][idx],
          yz = E.binv[5][idx];
  const T z[3] = {a * rr[0] + xy * rr[1] + xz * rr[2], xy * rr[0] + e * rr[1] + yz * rr[2],
                  xz * rr[0] + yz * rr[1] + f * rr[2]};
  const T* in[3] = {in0, in1, in2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T dd, xn;
    if (EPI == EPI_CHEB1) {
      dd = (T)E.c0 * z[c];
      xn = in[c][idx] + dd;
    } else {
      dd = (T)E.c1 * in[c][idx] + (T)E.c2 * z[c];
      xn = E.xacc[c][idx] + dd;
    }
    E.r[c][idx] = rr[c];
    E.dout[c][idx] = dd;
    E.xout[c][idx] = xn;
  }
}

// EK: viscosity storage (TN_ETA_F32: eta.v; TN_ETA_BF16 / TN_ETA_F16: eta.q times eta.cs, the
// column factor folded into |det M| once per column).
// A CTA owns TI x TJ lateral node columns and computes the (TI + 1) x (TJ + 1) cells touching them.
#define TN_TILE_PARAMS                                                                                          \
  Dims D, Op op, const T *__restrict__ in0, const T *__restrict__ in1, const T *__restrict__ in2,             \
      const T *__restrict__ in3, T *__restrict__ out0, T *__restrict__ out1, T *__restrict__ out2, const T *__restrict__ geo,             \
      const T *__restrict__ lay, EtaView<T> eta, const T *__restrict__ svec, int bc_in, int bc_out, int kc,    \
      const int *__restrict__ skip, EpiArgs<T> E
#define TN_TILE_ARGS D, op, in0, in1, in2, in3, out0, out1, out2, geo, lay, eta, svec, bc_in, bc_out, kc, skip, E
// Shared memory of a tile: NS per-node values (corner sums s and, for ops that need them,
// differences d of the input, per component) on the (TI + 2) x (TJ + 2) nodes the cells touch,
// then corners 10, 01, 11 of every cell's output contributions.
template <typename T, typename Op, int TI, int TJ>
struct TileSmem {
  // FP64 shares the per-node sums through shared memory (the FP64 pipe is the bottleneck); the
  // issue-bound FP32 kernels form them per cell from four corner loads instead (measured faster)
  static constexpr bool SHARE = sizeof(T) == 8;
  static constexpr int NS = (Op::LOADS && SHARE) ? (Op::NEEDS_D ? 2 * Op::NIN : Op::NIN) : 0;
  static constexpr int SD = NS * (TI + 2) * (TJ + 2);
  static constexpr int SM = 3 * Op::NOUT * (TI + 1) * (TJ + 1);
  static constexpr size_t bytes = sizeof(T) * (size_t)(SD + SM);
};

template <typename T, typename Op, int TI, int TJ, int FLAGS, int EPI, int EK>
__device__ __forceinline__ void tile_body(TN_TILE_PARAMS) {
  // All offsets are 32-bit: launch_tile only accepts levels whose node and wedge arrays have
  // fewer than 2^31 entries.
  constexpr int NIN = Op::NIN, NOUT = Op::NOUT, WI = TI + 1, WJ = TJ + 1;
  using Sh = TileSmem<T, Op, TI, TJ>;
  constexpr int NS = Sh::NS;
  extern __shared__ __align__(16) unsigned char tile_smem[];
  T* const sd = reinterpret_cast<T*>(tile_smem);  // [NS][WI + 1][WJ + 1]
  T* const sm = sd + Sh::SD;                        // [3][NOUT][WI][WJ]
  auto SD = [&](int v, int i, int j) -> T& { return sd[(v * (WI + 1) + i) * (WJ + 1) + j]; };
  auto SM = [&](int q, int c, int i, int j) -> T& { return sm[((q * NOUT + c) * WI + i) * WJ + j]; };
  if (skip && *skip) return;  // device-side early exit (uniform over the grid)
  const int N = D.N, n_r = D.n_r, P = D.P;
  const int LS = (int)D.layer_stride, NLL = (int)D.n_lat_layout;
  const int ntj = N / TJ;
  const int i0 = (blockIdx.x / ntj) * TI, j0 = (blockIdx.x % ntj) * TJ;
  const int d = blockIdx.z;
  const int kc0 = blockIdx.y * kc, kc1 = min(n_r - 1, kc0 + kc);
  const int ti = threadIdx.x / WJ, tj = threadIdx.x % WJ;
  const int ci = i0 - 1 + ti, cj = j0 - 1 + tj;  // this thread's cell
  const bool cell_ok = ci >= 0 && cj >= 0;       // ci, cj <= N - 1 always
  const int ci0 = max(ci, 0), cj0 = max(cj, 0);
  // node offset of corner 00 of this cell on layer 0 (the thread's own node when cell_ok)
  const int c00 = (int)(d * D.diamond_stride) + ci0 * P + cj0;
  const int lat00 = d * (N + 1) * P + ci0 * P + cj0;  // lateral-layout offset of corner 00
  // per-cell lateral geometry (both triangles), kept in registers for the whole column
  T Mi[2][9], dM[2];
  {
    const int t0 = ((d * N + ci0) * N + cj0) * 2, nt = (int)D.n_tri;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
#pragma unroll
      for (int q = 0; q < 9; ++q) Mi[w][q] = geo[q * nt + t0 + w];
      dM[w] = geo[9 * nt + t0 + w];
      if (EK != TN_ETA_F32 && Op::USES_ETA) dM[w] *= eta.cs[t0 + w];
    }
  }
  const typename Op::Col col = op.column(Mi, dM, ((d * N + ci0) * N + cj0) * 2);
  // viscosity of the cell's two wedges at layer k: pair k N^2 2 + {0, 1} past the column base
  const int eta_c0 = (((d * (n_r - 1)) * N + ci0) * N + cj0) * 2;
  const int eta_ls = N * N * 2;
  // the node this thread owns: (ci, cj) when ti, tj >= 1; the last tile row / column also owns
  // node N (handled in the rare path below)
  const bool own = ti >= 1 && tj >= 1;
  const bool own_shared = ci == 0 || ci == N || cj == 0 || cj == N;
  const bool last_i = (i0 + TI == N) && ti == TI, last_j = (j0 + TJ == N) && tj == TJ;
  // when own, ci = ci0 and cj = cj0: the owned node is corner 00 (offsets c00 and lat00)

  // Input nodes: every thread reads its own node (ci, cj) (slot (ti, tj) of sd) and carries it
  // from layer to layer; the WI + WJ + 1 nodes of the extra row i0 + TI and column j0 + TJ
  // (slots WI and WJ) are read, both layers, by threads 0, 1, ... (extra_node).
  constexpr int NX = WI + WJ + 1;
  auto extra_node = [&](int e, int& si, int& sj) {
    si = e < WJ ? WI : (e < WJ + WI ? e - WJ : WI);
    sj = e < WJ ? e : WJ;
  };
  // load one node's input at layer k (projected at the boundary layers), zero if absent
  auto load_node = [&](bool ok, int off, int lat, int k, T (&v)[NIN]) {
#pragma unroll
    for (int c = 0; c < NIN; ++c) v[c] = (T)0;
    if (!ok) return;
    const int o = off + k * LS;
    v[0] = in0[o];
    if (NIN > 1) v[NIN > 1 ? 1 : 0] = in1[o];
    if (NIN > 2) v[NIN > 2 ? 2 : 0] = in2[o];
    if (NIN > 3) v[NIN > 3 ? 3 : 0] = in3[o];
    if ((FLAGS & PROJ_IN) && (k == 0 || k == n_r - 1)) {
      T vv[3] = {v[0], v[NIN > 1 ? 1 : 0], v[NIN > 2 ? 2 : 0]};
      project_vec(vv, svec, (int64_t)lat, (int64_t)NLL, k == 0 ? bc_in : bc_out);
#pragma unroll
      for (int c = 0; c < (NIN < 3 ? NIN : 3); ++c) v[c] = vv[c];
    }
  };
  // corner sums / differences of one node between layers k and k+1 into sd slot (i, j)
  auto put_node = [&](int i, int j, const T (&b)[NIN], const T (&t)[NIN], T (&sv)[NIN], T (&dv)[NIN]) {
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
      sv[c] = b[c] + t[c];
      SD(c, i, j) = sv[c];
      if (Op::NEEDS_D) {
        dv[c] = t[c] - b[c];
        SD(NIN + c, i, j) = dv[c];
      }
    }
  };

  // boundary epilogue and store of node value v at layout offset idx (lateral offset so)
  auto store_node = [&](int k, int idx, int so, bool shared, T (&v)[3]) {
    if ((FLAGS & PROJ_OUT) && (k == 0 || k == n_r - 1)) {
      const int bc = k == 0 ? bc_in : bc_out;
      project_vec(v, svec, (int64_t)so, (int64_t)NLL, bc);
      if ((FLAGS & ADD_ID) && !shared) {
        T uu[3] = {in0[idx], in1[idx], in2[idx]};
        T pu[3] = {uu[0], uu[1], uu[2]};
        project_vec(pu, svec, (int64_t)so, (int64_t)NLL, bc);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += uu[c] - pu[c];
      }
    }
    if (EPI != EPI_NONE && !shared) {  // fused vector update; nothing else is stored
      epilogue<T, EPI>(E, in0, in1, in2, idx, v);
      return;
    }
    out0[idx] = v[0];
    if (NOUT > 1) out1[idx] = v[NOUT > 1 ? 1 : 0];
    if (NOUT > 2) out2[idx] = v[NOUT > 2 ? 2 : 0];
  };

  // exchange the node-level sums of the four corners and write the owned nodes of layer k.  The
  // caller has synchronised since sm was last read; sd is not touched.
  auto exchange_write = [&](int k, const T (&acc)[4][NOUT]) {
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) SM(q - 1, c, ti, tj) = acc[q][c];
    __syncthreads();
    if (own) {
      // node (ci, cj): cell (ci, cj) corner 00 + (ci-1, cj) corner 10 + (ci, cj-1) corner 01 +
      // (ci-1, cj-1) corner 11, in that order
      T v[3] = {0, 0, 0};
#pragma unroll
      for (int c = 0; c < NOUT; ++c)
        v[c] = ((acc[0][c] + SM(0, c, ti - 1, tj)) + SM(1, c, ti, tj - 1)) + SM(2, c, ti - 1, tj - 1);
      store_node(k, c00 + k * LS, lat00, own_shared, v);
    }
    if (last_i || last_j) {  // rare: nodes in row / column N of the diamond
#pragma unroll
      for (int oi = 0; oi < 2; ++oi)
#pragma unroll
        for (int oj = 0; oj < 2; ++oj) {
          if (oi == 0 && oj == 0) continue;
          if (oi == 1 && !last_i) continue;
          if (oj == 1 && !last_j) continue;
          const int xi = ti + oi, xj = tj + oj;
          if (xi < 1 || xj < 1) continue;
          const int ni = ci + oi, nj = cj + oj;
          // node (ni, nj) is in row or column N: no cell has it as corner 00
          T v[3] = {0, 0, 0};
#pragma unroll
          for (int c = 0; c < NOUT; ++c) {
            T b = (xj <= TJ) ? SM(0, c, xi - 1, xj) : (T)0;
            T e = (xi <= TI) ? SM(1, c, xi, xj - 1) : (T)0;
            T f = SM(2, c, xi - 1, xj - 1);
            v[c] = (b + e) + f;
          }
          const bool shared = ni == 0 || ni == N || nj == 0 || nj == N;
          store_node(k, (int)(d * D.diamond_stride) + k * LS + ni * P + nj, d * (N + 1) * P + ni * P + nj, shared,
                     v);
        }
    }
  };

  // per-cell path (FP32): the four corners of the cell, carried from layer to layer
  constexpr bool PERCELL = Op::LOADS && !Sh::SHARE;
  const int cdel[4] = {0, P, 1, P + 1};
  auto load_corners = [&](int k, T (&v)[4][NIN]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NIN; ++c) v[q][c] = (T)0;
    if (!cell_ok) return;
    const int o = c00 + k * LS;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q][0] = in0[o + cdel[q]];
      if (NIN > 1) v[q][NIN > 1 ? 1 : 0] = in1[o + cdel[q]];
      if (NIN > 2) v[q][NIN > 2 ? 2 : 0] = in2[o + cdel[q]];
      if (NIN > 3) v[q][NIN > 3 ? 3 : 0] = in3[o + cdel[q]];
    }
    if ((FLAGS & PROJ_IN) && (k == 0 || k == n_r - 1)) {
      const int bc = k == 0 ? bc_in : bc_out;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T vv[3] = {v[q][0], v[q][NIN > 1 ? 1 : 0], v[q][NIN > 2 ? 2 : 0]};
        project_vec(vv, svec, (int64_t)(lat00 + cdel[q]), (int64_t)NLL, bc);
#pragma unroll
        for (int c = 0; c < (NIN < 3 ? NIN : 3); ++c) v[q][c] = vv[c];
      }
    }
  };
  T ubc[PERCELL ? 4 : 1][NIN];

  T ub[NIN];  // own node at the bottom layer of the current cell layer
  T carry[4][NOUT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < NOUT; ++c) carry[q][c] = 0;

  const int kstart = kc0 > 0 ? kc0 - 1 : 0;
  if (NS > 0) load_node(cell_ok, c00, lat00, kstart, ub);
  if constexpr (PERCELL) load_corners(kstart, ubc);
  for (int k = kstart; k < kc1; ++k) {
    // corner sums and differences of layer pair (k, k+1): own node, then the extra nodes
    T s[4][NIN], dd[4][NIN];
    if constexpr (PERCELL) {
      T utc[4][NIN];
      load_corners(k + 1, utc);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NIN; ++c) {
          s[q][c] = ubc[q][c] + utc[q][c];
          if (Op::NEEDS_D) dd[q][c] = utc[q][c] - ubc[q][c];
          ubc[q][c] = utc[q][c];
        }
    }
    if (NS > 0) {
      T ut[NIN];
      load_node(cell_ok, c00, lat00, k + 1, ut);
      put_node(ti, tj, ub, ut, s[0], dd[0]);
#pragma unroll
      for (int c = 0; c < NIN; ++c) ub[c] = ut[c];
      for (int e = (int)threadIdx.x; e < NX; e += (int)blockDim.x) {
        int si, sj;
        extra_node(e, si, sj);
        const int ni = i0 - 1 + si, nj = j0 - 1 + sj;
        const bool ok = ni >= 0 && nj >= 0;  // ni, nj <= N always
        const int off = (int)(d * D.diamond_stride) + max(ni, 0) * P + max(nj, 0);
        const int lat = d * (N + 1) * P + max(ni, 0) * P + max(nj, 0);
        T xb[NIN], xt[NIN], xs[NIN], xd[NIN];
        load_node(ok, off, lat, k, xb);
        load_node(ok, off, lat, k + 1, xt);
        put_node(si, sj, xb, xt, xs, xd);
      }
      __syncthreads();
      // corners 10, 01, 11 of this cell: nodes (ci+1, cj), (ci, cj+1), (ci+1, cj+1)
      const int qi[3] = {ti + 1, ti, ti + 1}, qj[3] = {tj, tj + 1, tj + 1};
#pragma unroll
      for (int q = 1; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NIN; ++c) {
          s[q][c] = SD(c, qi[q - 1], qj[q - 1]);
          if (Op::NEEDS_D) dd[q][c] = SD(NIN + c, qi[q - 1], qj[q - 1]);
        }
    }
    // fused vector update: start fetching the owned node's epilogue operands into L1 now, so
    // their latency overlaps the cell arithmetic (the epilogue runs after the exchange)
    if (TN_EPI_PREFETCH && EPI != EPI_NONE && own && !own_shared && k >= kc0) {
      const int idx = c00 + k * LS;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (EPI == EPI_CHEB2) prefetch_l1(E.r[c] + idx), prefetch_l1(E.xacc[c] + idx);
        else prefetch_l1(E.b[c] + idx);
      }
      if (EPI != EPI_RESID)
#pragma unroll
        for (int q = 0; q < 6; ++q) prefetch_l1(E.binv[q] + idx);
    }
    T accb[4][NOUT], acct[4][NOUT];  // assigned by the op (zero for a halo cell outside the diamond)
    if (!cell_ok) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NOUT; ++c) accb[q][c] = acct[q][c] = 0;
    } else {
      T e[2] = {(T)1, (T)1};
      if (Op::USES_ETA) {
        const int o = eta_c0 + k * eta_ls;  // even: the pair is one aligned vector load
        if (EK == TN_ETA_F32) {
          if (sizeof(T) == 8) {
            const double2 p = *reinterpret_cast<const double2*>(eta.v + o);
            e[0] = (T)p.x, e[1] = (T)p.y;
          } else {
            const float2 p = *reinterpret_cast<const float2*>(eta.v + o);
            e[0] = (T)p.x, e[1] = (T)p.y;
          }
        } else {
          const uint32_t p = *reinterpret_cast<const uint32_t*>(eta.q + o);
          e[0] = (T)from16<EK>((uint16_t)(p & 0xffffu)), e[1] = (T)from16<EK>((uint16_t)(p >> 16));
        }
      }
      op.cell(s, dd, Mi, dM, lay + kLayerStride * k, e, accb, acct, col);
    }
    if (k >= kc0) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NOUT; ++c) accb[q][c] += carry[q][c];
      exchange_write(k, accb);
    }
    // sd and sm are rewritten only after every thread has passed the next barrier, which comes
    // after its reads of this layer; without shared inputs (NS = 0) a barrier closes the layer
    if (NS == 0 || k < kc0) __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) carry[q][c] = acct[q][c];
  }
  if (kc1 == n_r - 1) {
    __syncthreads();  // sm of the last layer has been read by every thread
    exchange_write(n_r - 1, carry);
  }
}

// ------------------------------------------------------------------------------------ halo-free tiles
// FP64 levels with N >= 32: a CTA of TI x TJ threads computes exactly its TI x TJ cells (no halo
// recompute, no idle lanes).  Nodes with all four cells in the tile are finished here; the nodes
// on the tile's edges (the tile lines i = m TI and j = n TJ) get one partial sum per tile in a
// ring buffer, summed in a fixed order and finished by k_ring_fix.  A tile-line node (i, j)
// written by a tile with first cell (i0, j0) goes to slot 2 bi + bj, bi = (i == i0),
// bj = (j == j0); its index within a diamond layer is ring_index(i, j).
struct RingDims {
  int TI, TJ, H, RC;  // tile shape, nodes on horizontal tile lines, all tile-line nodes
};
__host__ __device__ inline RingDims ring_dims(int N, int TI, int TJ) {
  RingDims r;
  r.TI = TI, r.TJ = TJ;
  r.H = (N / TI + 1) * (N + 1);
  r.RC = r.H + (N / TJ + 1) * (N - N / TI);
  return r;
}
__device__ __forceinline__ int ring_index(const RingDims& R, int N, int i, int j) {
  if (i % R.TI == 0) return (i / R.TI) * (N + 1) + j;
  return R.H + (j / R.TJ) * (N - N / R.TI) + (i - i / R.TI - 1);
}
// ring[((slot * ncomp + c) * n_r + k) * 10 * RC + d RC + rid]

// C is the compute type of the element arithmetic, the shared-memory sums and the carried
// partials: T itself, or double-float (dfl) for FP64 storage (values converted at load and store).
template <typename C, typename Op, int TI, int TJ>
struct TileSmemHF {
  static constexpr int NS = Op::LOADS ? (Op::NEEDS_D ? 2 * Op::NIN : Op::NIN) : 0;
  static constexpr int SD = NS * (TI + 1) * (TJ + 1);
  static constexpr int SM = 3 * Op::NOUT * TI * TJ;
  static constexpr size_t bytes = sizeof(C) * (size_t)(SD + SM);
};

// Ops whose contributions all have one sign (POSITIVE = true) let the tile kernel sum nodes with
// the double-word addition without the second TwoSum; the others use the accurate one.
template <typename Op, typename = void>
struct IsPositive : std::false_type {};
template <typename Op>
struct IsPositive<Op, std::void_t<decltype(Op::POSITIVE)>> : std::integral_constant<bool, Op::POSITIVE> {};
template <typename Op, typename = void>
struct IsPrefetch : std::false_type {};
template <typename Op>
struct IsPrefetch<Op, std::void_t<decltype(Op::PREFETCH)>> : std::integral_constant<bool, Op::PREFETCH> {};
template <typename Op, typename C>
__device__ __forceinline__ C node_add(const C& a, const C& b) {
  if constexpr (std::is_same<C, dfl>::value && IsPositive<Op>::value) return add_nc(a, b);
  else return a + b;
}

// storage <-> compute conversions: identities, or binary64 <-> double-float
template <typename C>
__device__ __forceinline__ C to_compute(double x) {
  if constexpr (std::is_same<C, dfl>::value) return split(x);
  else return (C)x;
}
template <typename C>
__device__ __forceinline__ C to_compute(float x) {
  return (C)x;
}
template <typename T, typename C>
__device__ __forceinline__ T to_storage(const C& x) {
  if constexpr (std::is_same<C, dfl>::value) return (T)join(x);
  else return (T)x;
}

template <typename T, typename Op, int TI, int TJ, int FLAGS, int EPI, int EK, typename C = T>
__device__ __forceinline__ void tile_body_hf(TN_TILE_PARAMS, T* __restrict__ ring) {
  constexpr int NIN = Op::NIN, NOUT = Op::NOUT;
  using Sh = TileSmemHF<C, Op, TI, TJ>;
  constexpr int NS = Sh::NS;
  extern __shared__ __align__(16) unsigned char tile_smem[];
  C* const sd = reinterpret_cast<C*>(tile_smem);  // [NS][TI + 1][TJ + 1]
  C* const sm = sd + Sh::SD;                        // [3][NOUT][TI][TJ]
  auto SD = [&](int v, int i, int j) -> C& { return sd[(v * (TI + 1) + i) * (TJ + 1) + j]; };
  auto SM = [&](int q, int c, int i, int j) -> C& { return sm[((q * NOUT + c) * TI + i) * TJ + j]; };
  // the layer table in the compute type (for dfl the launcher passes the level's double-float copy)
  const C* const layc = reinterpret_cast<const C*>(lay);
  if (skip && *skip) return;
  const int N = D.N, n_r = D.n_r, P = D.P;
  const int LS = (int)D.layer_stride, NLL = (int)D.n_lat_layout;
  const RingDims RD = ring_dims(N, TI, TJ);
  const int ntj = N / TJ;
  const int i0 = (blockIdx.x / ntj) * TI, j0 = (blockIdx.x % ntj) * TJ;
  const int d = blockIdx.z;
  const int kc0 = blockIdx.y * kc, kc1 = min(n_r - 1, kc0 + kc);
  const int ti = threadIdx.x / TJ, tj = threadIdx.x % TJ;
  const int ci = i0 + ti, cj = j0 + tj;  // this thread's cell; its corner 00 is its own node
  const int c00 = (int)(d * D.diamond_stride) + ci * P + cj;
  const int lat00 = d * (N + 1) * P + ci * P + cj;
  C Mi[2][9], dM[2];
  {
    const int t0 = ((d * N + ci) * N + cj) * 2, nt = (int)D.n_tri;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
#pragma unroll
      for (int q = 0; q < 9; ++q) Mi[w][q] = to_compute<C>(geo[q * nt + t0 + w]);
      T dm = geo[9 * nt + t0 + w];
      if (EK != TN_ETA_F32 && Op::USES_ETA) dm *= eta.cs[t0 + w];
      dM[w] = to_compute<C>(dm);
    }
  }
  const typename Op::Col col = op.column(Mi, dM, ((d * N + ci) * N + cj) * 2);
  const int eta_c0 = (((d * (n_r - 1)) * N + ci) * N + cj) * 2;
  const int eta_ls = N * N * 2;
  const bool interior = ti >= 1 && tj >= 1;  // own node finished here (never on a diamond edge)

  // extra nodes (input sums and output partials): e < TJ + 1: row node (TI, e); then column
  // node (e - TJ - 1, TJ); threads 0 .. NX - 1
  constexpr int NX = TI + TJ + 1;
  auto extra_node = [&](int e, int& si, int& sj) {
    si = e <= TJ ? TI : e - TJ - 1;
    sj = e <= TJ ? e : TJ;
  };
  // a node's input values at layer k: load_raw issues the loads, finish_node projects them on the
  // boundary layers and converts them to the compute type (load_node does both at once)
  auto load_raw = [&](int off, int k, T (&v)[NIN]) {
    const int o = off + k * LS;
    v[0] = in0[o];
    if (NIN > 1) v[NIN > 1 ? 1 : 0] = in1[o];
    if (NIN > 2) v[NIN > 2 ? 2 : 0] = in2[o];
    if (NIN > 3) v[NIN > 3 ? 3 : 0] = in3[o];
  };
  auto finish_node = [&](int lat, int k, T (&v)[NIN], C (&vc)[NIN]) {
    if ((FLAGS & PROJ_IN) && (k == 0 || k == n_r - 1)) {
      T vv[3] = {v[0], v[NIN > 1 ? 1 : 0], v[NIN > 2 ? 2 : 0]};
      project_vec(vv, svec, (int64_t)lat, (int64_t)NLL, k == 0 ? bc_in : bc_out);
#pragma unroll
      for (int c = 0; c < (NIN < 3 ? NIN : 3); ++c) v[c] = vv[c];
    }
#pragma unroll
    for (int c = 0; c < NIN; ++c) vc[c] = to_compute<C>(v[c]);
  };
  auto load_node = [&](int off, int lat, int k, C (&vc)[NIN]) {
    T v[NIN];
    load_raw(off, k, v);
    finish_node(lat, k, v, vc);
  };
  auto put_node = [&](int i, int j, const C (&b)[NIN], const C (&t)[NIN], C (&sv)[NIN], C (&dv)[NIN]) {
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
      sv[c] = b[c] + t[c];
      SD(c, i, j) = sv[c];
      if (Op::NEEDS_D) {
        dv[c] = t[c] - b[c];
        SD(NIN + c, i, j) = dv[c];
      }
    }
  };
  auto store_node = [&](int k, int idx, int so, const C (&vc)[3]) {  // a finished node off the diamond edges
    T v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = c < NOUT ? to_storage<T>(vc[c]) : (T)0;
    if ((FLAGS & PROJ_OUT) && (k == 0 || k == n_r - 1)) {
      const int bc = k == 0 ? bc_in : bc_out;
      project_vec(v, svec, (int64_t)so, (int64_t)NLL, bc);
      if (FLAGS & ADD_ID) {
        T uu[3] = {in0[idx], in1[idx], in2[idx]};
        T pu[3] = {uu[0], uu[1], uu[2]};
        project_vec(pu, svec, (int64_t)so, (int64_t)NLL, bc);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += uu[c] - pu[c];
      }
    }
    if (EPI != EPI_NONE) {
      epilogue<T, EPI>(E, in0, in1, in2, idx, v);
      return;
    }
    out0[idx] = v[0];
    if (NOUT > 1) out1[idx] = v[NOUT > 1 ? 1 : 0];
    if (NOUT > 2) out2[idx] = v[NOUT > 2 ? 2 : 0];
  };
  const int64_t ring_c = (int64_t)n_r * 10 * RD.RC;  // stride of one (slot, component)
  auto ring_store = [&](int k, int i, int j, int slot, const C (&v)[3]) {
    const int64_t base = (int64_t)k * 10 * RD.RC + (int64_t)d * RD.RC + ring_index(RD, N, i, j);
#pragma unroll
    for (int c = 0; c < NOUT; ++c) ring[(slot * NOUT + c) * ring_c + base] = to_storage<T>(v[c]);
  };
  auto exchange_write = [&](int k, const C (&acc)[4][NOUT]) {
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) SM(q - 1, c, ti, tj) = acc[q][c];
    __syncthreads();
    {
      // own node (ci, cj): this cell's corner 00 + (ci-1, cj) corner 10 + (ci, cj-1) corner 01 +
      // (ci-1, cj-1) corner 11, the cells of this tile only
      C v[3] = {C(0.0), C(0.0), C(0.0)};
#pragma unroll
      for (int c = 0; c < NOUT; ++c) {
        C a = acc[0][c];
        if (ti >= 1) a = node_add<Op>(a, SM(0, c, ti - 1, tj));
        if (tj >= 1) a = node_add<Op>(a, SM(1, c, ti, tj - 1));
        if (ti >= 1 && tj >= 1) a = node_add<Op>(a, SM(2, c, ti - 1, tj - 1));
        v[c] = a;
      }
      if (interior) store_node(k, c00 + k * LS, lat00, v);
      else ring_store(k, ci, cj, 2 * (ti == 0) + (tj == 0), v);
    }
    for (int e = (int)threadIdx.x; e < NX; e += (int)blockDim.x) {
      int si, sj;
      extra_node(e, si, sj);
      // node (i0 + si, j0 + sj) on the far row / column: cells (si - 1, sj) corner 10,
      // (si, sj - 1) corner 01, (si - 1, sj - 1) corner 11 where they are in the tile
      C v[3] = {C(0.0), C(0.0), C(0.0)};
#pragma unroll
      for (int c = 0; c < NOUT; ++c) {
        C a = C(0.0);
        if (si >= 1 && sj < TJ) a = node_add<Op>(a, SM(0, c, si - 1, sj));
        if (sj >= 1 && si < TI) a = node_add<Op>(a, SM(1, c, si, sj - 1));
        if (si >= 1 && sj >= 1) a = node_add<Op>(a, SM(2, c, si - 1, sj - 1));
        v[c] = a;
      }
      ring_store(k, i0 + si, j0 + sj, 2 * (si == 0) + (sj == 0), v);
    }
  };

  C ub[NIN];
  C carry[4][NOUT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < NOUT; ++c) carry[q][c] = C(0.0);
  const int kstart = kc0 > 0 ? kc0 - 1 : 0;
  // PREFETCH ops (light element work, held by load latency): the raw input of node layer k + 2 is
  // loaded while cell layer k is computed, and the extra node (one per thread < NX) keeps its
  // bottom values from the previous layer instead of loading them again
  constexpr bool PF = IsPrefetch<Op>::value && NS > 0;
  T rawn[PF ? NIN : 1], rawx[PF ? NIN : 1];
  C xbot[PF ? NIN : 1];
  int xoff = 0, xlat = 0, xsi = 0, xsj = 0;
  const bool hasx = (int)threadIdx.x < NX;  // blockDim.x = TI TJ > NX
  if (hasx) {
    extra_node((int)threadIdx.x, xsi, xsj);
    const int ni = i0 + xsi, nj = j0 + xsj;  // <= N
    xoff = (int)(d * D.diamond_stride) + ni * P + nj;
    xlat = d * (N + 1) * P + ni * P + nj;
  }
  if (NS > 0) load_node(c00, lat00, kstart, ub);
  if constexpr (PF) {
    load_raw(c00, kstart + 1, rawn);
    if (hasx) {
      load_node(xoff, xlat, kstart, xbot);
      load_raw(xoff, kstart + 1, rawx);
    }
  }
  for (int k = kstart; k < kc1; ++k) {
    C s[4][NIN], dd[4][NIN];
    if constexpr (PF) {
      C ut[NIN];
      finish_node(lat00, k + 1, rawn, ut);
      if (k + 2 <= kc1) load_raw(c00, k + 2, rawn);
      put_node(ti, tj, ub, ut, s[0], dd[0]);
#pragma unroll
      for (int c = 0; c < NIN; ++c) ub[c] = ut[c];
      if (hasx) {
        C xt[NIN], xs[NIN], xd[NIN];
        finish_node(xlat, k + 1, rawx, xt);
        if (k + 2 <= kc1) load_raw(xoff, k + 2, rawx);
        put_node(xsi, xsj, xbot, xt, xs, xd);
#pragma unroll
        for (int c = 0; c < NIN; ++c) xbot[c] = xt[c];
      }
      __syncthreads();
    } else if (NS > 0) {
      C ut[NIN];
      load_node(c00, lat00, k + 1, ut);
      put_node(ti, tj, ub, ut, s[0], dd[0]);
#pragma unroll
      for (int c = 0; c < NIN; ++c) ub[c] = ut[c];
      if (hasx) {
        C xb[NIN], xt[NIN], xs[NIN], xd[NIN];
        load_node(xoff, xlat, k, xb);
        load_node(xoff, xlat, k + 1, xt);
        put_node(xsi, xsj, xb, xt, xs, xd);
      }
      __syncthreads();
    }
    if (NS > 0) {
      const int qi[3] = {ti + 1, ti, ti + 1}, qj[3] = {tj, tj + 1, tj + 1};
#pragma unroll
      for (int q = 1; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NIN; ++c) {
          s[q][c] = SD(c, qi[q - 1], qj[q - 1]);
          if (Op::NEEDS_D) dd[q][c] = SD(NIN + c, qi[q - 1], qj[q - 1]);
        }
    }
    if (TN_EPI_PREFETCH && EPI != EPI_NONE && interior && k >= kc0) {
      const int idx = c00 + k * LS;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (EPI == EPI_CHEB2) prefetch_l1(E.r[c] + idx), prefetch_l1(E.xacc[c] + idx);
        else prefetch_l1(E.b[c] + idx);
      }
      if (EPI != EPI_RESID)
#pragma unroll
        for (int q = 0; q < 6; ++q) prefetch_l1(E.binv[q] + idx);
    }
    C accb[4][NOUT], acct[4][NOUT];
    {
      C e[2] = {C(1.0), C(1.0)};
      if (Op::USES_ETA) {
        const int o = eta_c0 + k * eta_ls;
        if (EK == TN_ETA_F32) {
          const double2 p = *reinterpret_cast<const double2*>(eta.v + o);
          e[0] = to_compute<C>((T)p.x), e[1] = to_compute<C>((T)p.y);
        } else {
          const uint32_t p = *reinterpret_cast<const uint32_t*>(eta.q + o);
          e[0] = C(from16<EK>((uint16_t)(p & 0xffffu))), e[1] = C(from16<EK>((uint16_t)(p >> 16)));
        }
      }
      op.cell(s, dd, Mi, dM, layc + kLayerStride * k, e, accb, acct, col);
    }
    if (k >= kc0) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NOUT; ++c) accb[q][c] = node_add<Op>(accb[q][c], carry[q][c]);
      exchange_write(k, accb);
    }
    if (NS == 0 || k < kc0) __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) carry[q][c] = acct[q][c];
  }
  if (kc1 == n_r - 1) {
    __syncthreads();
    exchange_write(n_r - 1, carry);
  }
}

// Halo-free FP64 tiles: TI x TJ threads, one CTA per SM.
template <typename T, typename Op, int TI, int TJ, int FLAGS, int EPI = EPI_NONE, int EK = TN_ETA_F32,
          typename C = T>
__global__ void __launch_bounds__(TI * TJ, 1) k_tile_hf(TN_TILE_PARAMS, T* __restrict__ ring) {
  tile_body_hf<T, Op, TI, TJ, FLAGS, EPI, EK, C>(TN_TILE_ARGS, ring);
}

// Thread per tile-line node and layer: the fixed-order sum of the tiles' partials (slots 0..3 of
// the tiles that exist around the node), then the node is finished like in the tile kernel:
// diamond-edge nodes get the diamond's partial sum (projected) for the interface pass.
template <typename T, int NOUT, int FLAGS, int EPI>
__global__ void k_ring_fix(Dims D, RingDims RD, const T* __restrict__ ring, const T* __restrict__ in0,
                           const T* __restrict__ in1, const T* __restrict__ in2, T* __restrict__ out0,
                           T* __restrict__ out1, T* __restrict__ out2, const T* __restrict__ svec, int bc_in,
                           int bc_out, const int* __restrict__ skip, EpiArgs<T> E) {
  if (skip && *skip) return;
  const int N = D.N, n_r = D.n_r;
  const int rid = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y, d = blockIdx.z;  // grid: RC x n_r x 10
  if (rid >= RD.RC) return;
  const int64_t per_k = (int64_t)10 * RD.RC;
  int i, j;
  if (rid < RD.H) {
    i = (rid / (N + 1)) * RD.TI, j = rid % (N + 1);
  } else {
    const int r2 = rid - RD.H, per = N - N / RD.TI;
    const int t = r2 % per;
    j = (r2 / per) * RD.TJ;
    i = (t / (RD.TI - 1)) * RD.TI + 1 + t % (RD.TI - 1);
  }
  const bool on_h = i % RD.TI == 0, on_v = j % RD.TJ == 0;
  const int64_t ring_c = (int64_t)n_r * 10 * RD.RC;
  const int64_t base = (int64_t)k * per_k + (int64_t)d * RD.RC + rid;
  T v[3] = {0, 0, 0};
  for (int bi = 0; bi < 2; ++bi) {
    if (bi == 1 && !on_h) break;
    if (on_h && ((bi == 0 && i == 0) || (bi == 1 && i == N))) continue;  // no tile there
    for (int bj = 0; bj < 2; ++bj) {
      if (bj == 1 && !on_v) break;
      if (on_v && ((bj == 0 && j == 0) || (bj == 1 && j == N))) continue;
      const int slot = 2 * bi + bj;
#pragma unroll
      for (int c = 0; c < NOUT; ++c) v[c] += ring[(slot * NOUT + c) * ring_c + base];
    }
  }
  const int M = N + 1;
  const int idx = (int)(d * D.diamond_stride) + k * (int)D.layer_stride + i * D.P + j;
  const int64_t so = ((int64_t)d * M + i) * D.P + j;
  const bool shared = i == 0 || i == N || j == 0 || j == N;
  if ((FLAGS & PROJ_OUT) && (k == 0 || k == n_r - 1)) {
    const int bc = k == 0 ? bc_in : bc_out;
    project_vec(v, svec, so, D.n_lat_layout, bc);
    if ((FLAGS & ADD_ID) && !shared) {
      T uu[3] = {in0[idx], in1[idx], in2[idx]};
      T pu[3] = {uu[0], uu[1], uu[2]};
      project_vec(pu, svec, so, D.n_lat_layout, bc);
      for (int c = 0; c < 3; ++c) v[c] += uu[c] - pu[c];
    }
  }
  if (EPI != EPI_NONE && !shared) {
    epilogue<T, EPI>(E, in0, in1, in2, idx, v);
    return;
  }
  out0[idx] = v[0];
  if (NOUT > 1) out1[idx] = v[NOUT > 1 ? 1 : 0];
  if (NOUT > 2) out2[idx] = v[NOUT > 2 ? 2 : 0];
}

#include "pair32.cuh"

// Square tiles: MinBlocks CTAs per SM through the register cap of the launch bounds.
template <typename T, typename Op, int TI, int TJ, int FLAGS, int EPI = EPI_NONE, int EK = TN_ETA_F32>
__global__ void __launch_bounds__((TI + 1) * (TJ + 1), MinBlocks<T>::value) k_tile(TN_TILE_PARAMS) {
  tile_body<T, Op, TI, TJ, FLAGS, EPI, EK>(TN_TILE_ARGS);
}

// Wide tiles (16 x 32 nodes, 561 threads, one CTA per SM): registers capped at TN_WIDE_MAXREG so
// that the CTA fits the register file.
template <typename T, typename Op, int TI, int TJ, int FLAGS, int EPI = EPI_NONE, int EK = TN_ETA_F32>
__global__ void __maxnreg__(TN_WIDE_MAXREG) k_tile_wide(TN_TILE_PARAMS) {
  tile_body<T, Op, TI, TJ, FLAGS, EPI, EK>(TN_TILE_ARGS);
}

// Compute type of an op's element arithmetic: the storage type, except for the double-float
// viscous ops on FP64 data.
template <typename Op, typename T>
struct OpCompute {
  using type = T;
};
template <bool HG, typename T>
struct OpCompute<OpA<dfl, HG>, T> {
  using type = dfl;
};
template <bool RHO, typename T>
struct OpCompute<OpDiv<dfl, RHO>, T> {
  using type = dfl;
};
template <typename T>
struct OpCompute<OpGrad<dfl>, T> {
  using type = dfl;
};
template <bool HG, typename T>
struct OpCompute<OpDiag<dfl, HG>, T> {
  using type = dfl;
};

template <typename T, typename Op, int FLAGS, int EPI = EPI_NONE>
cudaError_t launch_tile(const Level& L, BC bc, Op op, const T* const* in, T* const* out, const EtaView<T>& eta,
                        cudaStream_t st, const int* skip = nullptr, const EpiArgs<T>* epi = nullptr) {
  // double-float ops exist for the halo-free FP64 tiles only (levels with N >= 32)
  using C = typename OpCompute<Op, T>::type;
  constexpr bool kDF = !std::is_same<C, T>::value;
  EpiArgs<T> E{};
  if (epi) E = *epi;
  Dims D = dims(L);
  if (L.n_layout >= (int64_t)INT32_MAX || L.n_wedges >= (int64_t)INT32_MAX || 10 * L.n_tri >= (int64_t)INT32_MAX)
    return cudaErrorInvalidValue;  // the tile kernel uses 32-bit offsets
  // tile shape: FP64 16 x 32 nodes where N >= 32 (fewer halo cells and idle lanes per owned node,
  // one CTA per SM; measured slower for the issue-bound FP32 kernels), else square N' x N' with
  // N' = min(N, 16)
  constexpr bool kWideT = sizeof(T) == 8 && TN_WIDE_TILES;
  const bool wide = kWideT && L.N >= 2 * TILE;
  const int ti_ = L.N >= TILE ? TILE : L.N, tj_ = wide ? 2 * TILE : ti_;
  const int ntiles = (L.N / ti_) * (L.N / tj_);
  const int ncells = L.n_r - 1;
  // radial chunks: enough CTAs to fill the GPU a few times over (wide tiles: one CTA per SM)
  const int64_t target = wide ? TN_CTA_TARGET_WIDE : TN_CTA_TARGET;
  int kc = ncells;
  while (kc > TN_KC_MIN && (int64_t)ntiles * 10 * ((ncells + kc - 1) / kc) < target) kc = (kc + 1) / 2;
  dim3 grid(ntiles, (ncells + kc - 1) / kc, 10);
  const T* i1 = Op::NIN > 1 ? in[1] : in[0];
  const T* i2 = Op::NIN > 2 ? in[2] : in[0];
  const T* i3 = Op::NIN > 3 ? in[3] : in[0];
  T* o1 = Op::NOUT > 1 ? out[1] : out[0];
  T* o2 = Op::NOUT > 2 ? out[2] : out[0];
  const T* sv = Tab<T>::s(L);
  const T* geo = Tab<T>::geo(L);
  const T* lay = Tab<T>::lay(L);
  // kernels with more than 48 KB of shared memory (FP64 A on wide tiles) got their attribute
  // from prepare_tile_kernels() when the first mesh was created
#define TN_TILE_LAUNCH(KERNEL, TIv, TJv, EKv)                                                                   \
  KERNEL<T, Op, TIv, TJv, FLAGS, EPI, EKv><<<grid, (TIv + 1) * (TJv + 1), TileSmem<T, Op, TIv, TJv>::bytes, st>>>( \
      D, op, in[0], i1, i2, i3, out[0], o1, o2, geo, lay, eta, sv, bc.in, bc.out, kc, skip, E)
  // 16-bit viscosity (FP32 path only): only full tiles (levels with N >= 16 store it)
  if constexpr (Op::USES_ETA && sizeof(T) == 4) {
    if (eta.kind != TN_ETA_F32) {
      if (ti_ != TILE) return cudaErrorInvalidValue;
      if (eta.kind == TN_ETA_BF16) TN_TILE_LAUNCH(k_tile, TILE, TILE, TN_ETA_BF16);
      else TN_TILE_LAUNCH(k_tile, TILE, TILE, TN_ETA_F16);
      return cudaGetLastError();
    }
  }
  if constexpr (kDF) {
    if (!(wide && TN_HALO_FREE) || !L.laydf) return cudaErrorInvalidValue;
  }
  if constexpr (kWideT) {
    if (wide && TN_HALO_FREE) {
      // halo-free tiles: grid over the tiles proper, then the tile-line nodes
      if (!L.ring64) return cudaErrorInvalidValue;  // allocated with the level
      constexpr int TI = TILE, TJ = 2 * TILE;
      // the layer table in the compute type: the level's double-float copy for dfl ops
      const T* layk = kDF ? reinterpret_cast<const T*>(L.laydf) : lay;
      k_tile_hf<T, Op, TI, TJ, FLAGS, EPI, TN_ETA_F32, C><<<grid, TI * TJ, TileSmemHF<C, Op, TI, TJ>::bytes, st>>>(
          D, op, in[0], i1, i2, i3, out[0], o1, o2, geo, layk, eta, sv, bc.in, bc.out, kc, skip, E, (T*)L.ring64);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      const RingDims RD = ring_dims(L.N, TI, TJ);
      k_ring_fix<T, Op::NOUT, FLAGS, EPI><<<dim3(nblk(RD.RC, 256), L.n_r, 10), 256, 0, st>>>(D, RD, (const T*)L.ring64, in[0], i1, i2,
                                                                        out[0], o1, o2, sv, bc.in, bc.out, skip, E);
      return cudaGetLastError();
    }
    if constexpr (!kDF) {
      if (wide) {
        TN_TILE_LAUNCH(k_tile_wide, TILE, 2 * TILE, TN_ETA_F32);
        return cudaGetLastError();
      }
    }
  }
  if constexpr (!kDF) {
    switch (ti_) {
      case 16: TN_TILE_LAUNCH(k_tile, 16, 16, TN_ETA_F32); break;
      case 8: TN_TILE_LAUNCH(k_tile, 8, 8, TN_ETA_F32); break;
      case 4: TN_TILE_LAUNCH(k_tile, 4, 4, TN_ETA_F32); break;
      case 2: TN_TILE_LAUNCH(k_tile, 2, 2, TN_ETA_F32); break;
      case 1: TN_TILE_LAUNCH(k_tile, 1, 1, TN_ETA_F32); break;
      default:
        return cudaErrorInvalidValue;
    }
  }
#undef TN_TILE_LAUNCH
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------ interface
template <typename T>
__global__ void k_interface(Dims D, int n_groups, const int* __restrict__ gptr, const int64_t* __restrict__ goff,
                            const T* __restrict__ gs, int ncomp, int mode, T* y0, T* y1, T* y2,
                            const T* __restrict__ u0, const T* __restrict__ u1, const T* __restrict__ u2,
                            int bc_in, int bc_out, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;  // grid: groups x layers
  if (g >= n_groups) return;
  T* y[3] = {y0, y1, y2};
  const T* u[3] = {u0, u1, u2};
  const int b = gptr[g], e = gptr[g + 1];
  const int64_t lo = (int64_t)k * D.layer_stride;
  T v[3] = {0, 0, 0};
  for (int q = b; q < e; ++q)
    for (int c = 0; c < ncomp; ++c) v[c] += y[c][goff[q] + lo];
  if (mode != 0 && (k == 0 || k == D.n_r - 1)) {
    const int bc = k == 0 ? bc_in : bc_out;
    T w[3];
    if (mode == 1)
      for (int c = 0; c < 3; ++c) w[c] = u[c][goff[b] + lo];
    if (bc == TN_BC_NOSLIP) {
      for (int c = 0; c < 3; ++c) v[c] += mode == 1 ? w[c] : (T)1;
    } else {
      T s[3] = {gs[g], gs[n_groups + g], gs[2 * n_groups + g]};
      if (mode == 1) {
        T dot = w[0] * s[0] + w[1] * s[1] + w[2] * s[2];
        for (int c = 0; c < 3; ++c) v[c] += dot * s[c];
      } else {
        for (int c = 0; c < 3; ++c) v[c] += s[c] * s[c];
      }
    }
  }
  for (int q = b; q < e; ++q)
    for (int c = 0; c < ncomp; ++c) y[c][goff[q] + lo] = v[c];
}

// Interface sum of K x partials (mode 1: + (I - P) x at boundary layers) followed by the fused
// vector update of the group's node, written to every copy.
template <typename T, int EPI>
__global__ void k_interface_epi(Dims D, int n_groups, const int* __restrict__ gptr, const int64_t* __restrict__ goff,
                                const T* __restrict__ gs, const T* __restrict__ t0, const T* __restrict__ t1,
                                const T* __restrict__ t2, const T* __restrict__ x0, const T* __restrict__ x1,
                                const T* __restrict__ x2, int bc_in, int bc_out, const int* __restrict__ skip,
                                EpiArgs<T> E) {
  if (skip && *skip) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;  // grid: groups x layers
  if (g >= n_groups) return;
  const T* y[3] = {t0, t1, t2};
  const T* u[3] = {x0, x1, x2};
  const int b = gptr[g], e = gptr[g + 1];
  const int64_t lo = (int64_t)k * D.layer_stride;
  T v[3] = {0, 0, 0};
  for (int q = b; q < e; ++q)
    for (int c = 0; c < 3; ++c) v[c] += y[c][goff[q] + lo];
  if (k == 0 || k == D.n_r - 1) {
    const int bc = k == 0 ? bc_in : bc_out;
    T w[3];
    for (int c = 0; c < 3; ++c) w[c] = u[c][goff[b] + lo];
    if (bc == TN_BC_NOSLIP) {
      for (int c = 0; c < 3; ++c) v[c] += w[c];
    } else {
      T s[3] = {gs[g], gs[n_groups + g], gs[2 * n_groups + g]};
      T dot = w[0] * s[0] + w[1] * s[1] + w[2] * s[2];
      for (int c = 0; c < 3; ++c) v[c] += dot * s[c];
    }
  }
  for (int q = b; q < e; ++q) epilogue<T, EPI>(E, x0, x1, x2, (int)(goff[q] + lo), v);
}

// ------------------------------------------------------------------------------------ diag(A)
// Thread per layout node; gathers the 3x3 node block of A from the (up to) 12 wedges
// around the node: A_jj = sum_e V eta (|g|^2 I + 1/3 g g^T) (the -2/3 div term gives
// -2/3 g g^T, the symmetric-gradient term g g^T, so 1/3 with div_term, 1 without).
// Only the two boundary node layers are handled here (the tile kernel with OpDiag writes the
// interior layers): blocks = 10 * 2 * (N+1)^2 threads, layer 0 and layer n_r - 1.
// Hourglass-control part of the node block of wedge-local lateral node a (side 0: the node is on
// the wedge's bottom layer): eps n_a (k9 - zeta / 3)^2 times the identity (see OpDiag).
template <typename T>
__device__ __forceinline__ T hg_node_diag(const T (&Mi)[9], T dM, T et, const T* lc, T hgk, int a, int side) {
  T l = 0, q = 0;
  for (int x = 0; x < 3; ++x) {
    const T s01 = Mi[x] + Mi[3 + x];
    l += s01 * s01 + Mi[x] * Mi[x] + Mi[3 + x] * Mi[3 + x];
    q += Mi[6 + x] * Mi[6 + x];
  }
  const T eps = (hgk * et) * (lc[5] * ((T)2 * dM * l) + lc[9] * ((T)6 * dM * q));
  const T kz = side == 0 ? lc[8] + (T)(1.0 / 3.0) : lc[8] - (T)(1.0 / 3.0);
  return eps * (a == 0 ? (T)2 : (T)5) * (kz * kz);
}

// Second radial quadrature point (see OpDiag2): the wedge adds ve / 3 (|g1|^2 I + c g1 g1^T) with
// g1 = w0 (l_a + m2 / 3) to the node block, the same for its bottom and top node.
template <typename T>
__device__ __forceinline__ void add_second_point(const T (&Mi)[9], T cxi, T ceta, T c2, T ve, T third, T& alpha,
                                                 T (&B)[6]) {
  T g[3];
  for (int x = 0; x < 3; ++x) g[x] = Mi[x] * cxi + Mi[3 + x] * ceta + Mi[6 + x] * c2;
  const T v3 = ve * (T)(1.0 / 3.0), tv = v3 * third;
  alpha += v3 * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  B[0] += tv * g[0] * g[0], B[1] += tv * g[1] * g[1], B[2] += tv * g[2] * g[2];
  B[3] += tv * g[0] * g[1], B[4] += tv * g[0] * g[2], B[5] += tv * g[1] * g[2];
}

template <typename T>
__global__ void k_diag_A(Dims D, const T* __restrict__ geo, const T* __restrict__ lay, EtaView<T> eta,
                         const T* __restrict__ svec, int bc_in, int bc_out, int div_term, T hgk, int nq, T* d0,
                         T* d1, T* d2) {
  const int N = D.N, M = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: lattice points x 2 layers x 10 diamonds
  if (t >= M * M) return;
  const int i = t / M, j = t - i * M, side_ = blockIdx.y, d = blockIdx.z;
  const int k = side_ == 0 ? 0 : D.n_r - 1;
  // (cell di, cell dj, wedge, local lateral node) of the six triangles around lattice node (i, j)
  const int tri[6][4] = {{0, 0, 0, 0}, {-1, 0, 0, 1}, {-1, 0, 1, 2}, {0, -1, 0, 2}, {0, -1, 1, 1}, {-1, -1, 1, 0}};
  const T gxi[3] = {-1, 1, 0}, geta[3] = {-1, 0, 1};
  const T third = div_term ? (T)(1.0 / 3.0) : (T)1;
  T B[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
  T alpha = 0;
  for (int q = 0; q < 6; ++q) {
    const int ci = i + tri[q][0], cj = j + tri[q][1], w = tri[q][2], a = tri[q][3];
    if (ci < 0 || cj < 0 || ci >= N || cj >= N) continue;
    const int64_t t = (((int64_t)d * N + ci) * N + cj) * 2 + w;
    T Mi[9];
    for (int r = 0; r < 9; ++r) Mi[r] = geo[(int64_t)r * D.n_tri + t];
    const T dM = geo[(int64_t)9 * D.n_tri + t];
    for (int side = 0; side < 2; ++side) {  // side 0: node is bottom of layer k; 1: top of layer k-1
      const int kk = side == 0 ? k : k - 1;
      if (kk < 0 || kk >= D.n_r - 1) continue;
      const T w0 = lay[kLayerStride * kk], w1 = lay[kLayerStride * kk + 1], vol = lay[kLayerStride * kk + 2];
      const T gz = side == 0 ? (T)-1 : (T)1;
      T g[3];
      for (int x = 0; x < 3; ++x) g[x] = Mi[x] * (w0 * gxi[a]) + Mi[3 + x] * (w0 * geta[a]) + Mi[6 + x] * (w1 * gz);
      const T et = eta_at(eta, ((((int64_t)d * (D.n_r - 1) + kk) * N + ci) * N + cj) * 2 + w, t);
      const T ve = vol * dM * et;
      if (hgk > (T)0) alpha += hg_node_diag(Mi, dM, et, lay + kLayerStride * kk, hgk, a, side);
      const T g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      alpha += ve * g2;
      const T tv = ve * third;
      B[0] += tv * g[0] * g[0], B[1] += tv * g[1] * g[1], B[2] += tv * g[2] * g[2];
      B[3] += tv * g[0] * g[1], B[4] += tv * g[0] * g[2], B[5] += tv * g[1] * g[2];
      if (nq == 2) add_second_point(Mi, w0 * gxi[a], w0 * geta[a], w0 * (T)(1.0 / 3.0), ve, third, alpha, B);
    }
  }
  T A[3][3] = {{alpha + B[0], B[3], B[4]}, {B[3], alpha + B[1], B[5]}, {B[4], B[5], alpha + B[2]}};
  T out[3] = {A[0][0], A[1][1], A[2][2]};
  const bool shared = i == 0 || i == N || j == 0 || j == N;
  if (k == 0 || k == D.n_r - 1) {
    const int bc = k == 0 ? bc_in : bc_out;
    const int64_t so = ((int64_t)d * M + i) * D.P + j;
    if (bc == TN_BC_NOSLIP) {
      out[0] = out[1] = out[2] = 0;
    } else {
      const T s[3] = {svec[so], svec[so + D.n_lat_layout], svec[so + 2 * D.n_lat_layout]};
      T Pm[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Pm[r][c] = (r == c ? (T)1 : (T)0) - s[r] * s[c];
      for (int c = 0; c < 3; ++c) {  // (P A P)_cc = sum_{a,b} P_ca A_ab P_bc
        T acc = 0;
        for (int a2 = 0; a2 < 3; ++a2)
          for (int b2 = 0; b2 < 3; ++b2) acc += Pm[c][a2] * A[a2][b2] * Pm[b2][c];
        out[c] = acc;
      }
    }
    if (!shared) {
      if (bc == TN_BC_NOSLIP) {
        out[0] += 1, out[1] += 1, out[2] += 1;
      } else {
        for (int c = 0; c < 3; ++c) out[c] += svec[so + c * D.n_lat_layout] * svec[so + c * D.n_lat_layout];
      }
    }
  }
  const int64_t idx = (int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride + (int64_t)i * D.P + j;
  d0[idx] = out[0], d1[idx] = out[1], d2[idx] = out[2];
}

// ------------------------------------------------------------------------------------ node blocks
// Thread per layout node: the 3x3 node block of the constrained operator, P_j A_jj P_j + I - P_j,
// as 6 entries (xx, yy, zz, xy, xz, yz).  Same gather as k_diag_A; nodes on diamond edges get
// P A_partial P per diamond and the identity part is added once by k_interface_block.
template <typename T>
__global__ void k_block_A(Dims D, const T* __restrict__ geo, const T* __restrict__ lay, EtaView<T> eta,
                          const T* __restrict__ svec, int bc_in, int bc_out, int div_term, T hgk, int nq, T* b0,
                          T* b1, T* b2, T* b3, T* b4, T* b5) {
  const int N = D.N, M = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: lattice points x n_r x 10 diamonds
  if (t >= M * M) return;
  const int i = t / M, j = t - i * M, k = blockIdx.y, d = blockIdx.z;
  const int tri[6][4] = {{0, 0, 0, 0}, {-1, 0, 0, 1}, {-1, 0, 1, 2}, {0, -1, 0, 2}, {0, -1, 1, 1}, {-1, -1, 1, 0}};
  const T gxi[3] = {-1, 1, 0}, geta[3] = {-1, 0, 1};
  const T third = div_term ? (T)(1.0 / 3.0) : (T)1;
  T B[6] = {0, 0, 0, 0, 0, 0};
  T alpha = 0;
  for (int q = 0; q < 6; ++q) {
    const int ci = i + tri[q][0], cj = j + tri[q][1], w = tri[q][2], a = tri[q][3];
    if (ci < 0 || cj < 0 || ci >= N || cj >= N) continue;
    const int64_t t = (((int64_t)d * N + ci) * N + cj) * 2 + w;
    T Mi[9];
    for (int r = 0; r < 9; ++r) Mi[r] = geo[(int64_t)r * D.n_tri + t];
    const T dM = geo[(int64_t)9 * D.n_tri + t];
    for (int side = 0; side < 2; ++side) {
      const int kk = side == 0 ? k : k - 1;
      if (kk < 0 || kk >= D.n_r - 1) continue;
      const T w0 = lay[kLayerStride * kk], w1 = lay[kLayerStride * kk + 1], vol = lay[kLayerStride * kk + 2];
      const T gz = side == 0 ? (T)-1 : (T)1;
      T g[3];
      for (int x = 0; x < 3; ++x) g[x] = Mi[x] * (w0 * gxi[a]) + Mi[3 + x] * (w0 * geta[a]) + Mi[6 + x] * (w1 * gz);
      const T et = eta_at(eta, ((((int64_t)d * (D.n_r - 1) + kk) * N + ci) * N + cj) * 2 + w, t);
      const T ve = vol * dM * et;
      if (hgk > (T)0) alpha += hg_node_diag(Mi, dM, et, lay + kLayerStride * kk, hgk, a, side);
      alpha += ve * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      const T tv = ve * third;
      B[0] += tv * g[0] * g[0], B[1] += tv * g[1] * g[1], B[2] += tv * g[2] * g[2];
      B[3] += tv * g[0] * g[1], B[4] += tv * g[0] * g[2], B[5] += tv * g[1] * g[2];
      if (nq == 2) add_second_point(Mi, w0 * gxi[a], w0 * geta[a], w0 * (T)(1.0 / 3.0), ve, third, alpha, B);
    }
  }
  T A[3][3] = {{alpha + B[0], B[3], B[4]}, {B[3], alpha + B[1], B[5]}, {B[4], B[5], alpha + B[2]}};
  const bool shared = i == 0 || i == N || j == 0 || j == N;
  if (k == 0 || k == D.n_r - 1) {
    const int bc = k == 0 ? bc_in : bc_out;
    const int64_t so = ((int64_t)d * M + i) * D.P + j;
    T Pm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    T s[3] = {0, 0, 0};
    if (bc != TN_BC_NOSLIP) {
      for (int c = 0; c < 3; ++c) s[c] = svec[so + c * D.n_lat_layout];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Pm[r][c] = (r == c ? (T)1 : (T)0) - s[r] * s[c];
    }
    T PA[3][3], PAP[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) PA[r][c] = Pm[r][0] * A[0][c] + Pm[r][1] * A[1][c] + Pm[r][2] * A[2][c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) PAP[r][c] = PA[r][0] * Pm[0][c] + PA[r][1] * Pm[1][c] + PA[r][2] * Pm[2][c];
    if (!shared)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) PAP[r][c] += bc == TN_BC_NOSLIP ? (r == c ? (T)1 : (T)0) : s[r] * s[c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) A[r][c] = PAP[r][c];
  }
  const int64_t idx = (int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride + (int64_t)i * D.P + j;
  b0[idx] = A[0][0], b1[idx] = A[1][1], b2[idx] = A[2][2], b3[idx] = A[0][1], b4[idx] = A[0][2], b5[idx] = A[1][2];
}

// Sum the 6 block entries over the copies of shared nodes; add I - P once at boundary layers.
template <typename T>
__global__ void k_interface_block(Dims D, int n_groups, const int* __restrict__ gptr, const int64_t* __restrict__ goff,
                                  const T* __restrict__ gs, T* b0, T* b1, T* b2, T* b3, T* b4, T* b5, int bc_in,
                                  int bc_out) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= (int64_t)n_groups * D.n_r) return;
  const int g = (int)(gid % n_groups), k = (int)(gid / n_groups);
  T* y[6] = {b0, b1, b2, b3, b4, b5};
  const int b = gptr[g], e = gptr[g + 1];
  const int64_t lo = (int64_t)k * D.layer_stride;
  T v[6] = {0, 0, 0, 0, 0, 0};
  for (int q = b; q < e; ++q)
    for (int c = 0; c < 6; ++c) v[c] += y[c][goff[q] + lo];
  if (k == 0 || k == D.n_r - 1) {
    const int bc = k == 0 ? bc_in : bc_out;
    if (bc == TN_BC_NOSLIP) {
      v[0] += 1, v[1] += 1, v[2] += 1;
    } else {
      const T s[3] = {gs[g], gs[n_groups + g], gs[2 * n_groups + g]};
      v[0] += s[0] * s[0], v[1] += s[1] * s[1], v[2] += s[2] * s[2];
      v[3] += s[0] * s[1], v[4] += s[0] * s[2], v[5] += s[1] * s[2];
    }
  }
  for (int q = b; q < e; ++q)
    for (int c = 0; c < 6; ++c) y[c][goff[q] + lo] = v[c];
}

// In place: symmetric 3x3 block (xx, yy, zz, xy, xz, yz) -> its inverse (0 where singular / padding).
template <typename T>
__global__ void k_block_inv(int64_t n, T* b0, T* b1, T* b2, T* b3, T* b4, T* b5) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T a = b0[i], e = b1[i], f = b2[i], bb = b3[i], c = b4[i], dd = b5[i];
  // [[a, bb, c], [bb, e, dd], [c, dd, f]]
  const T c00 = e * f - dd * dd, c01 = c * dd - bb * f, c02 = bb * dd - c * e;
  const T det = a * c00 + bb * c01 + c * c02;
  if (det == (T)0) {
    b0[i] = b1[i] = b2[i] = b3[i] = b4[i] = b5[i] = (T)0;
    return;
  }
  const T id = (T)1 / det;
  b0[i] = c00 * id;
  b1[i] = (a * f - c * c) * id;
  b2[i] = (a * e - bb * bb) * id;
  b3[i] = c01 * id;
  b4[i] = c02 * id;
  b5[i] = (bb * c - a * dd) * id;
}

// ------------------------------------------------------------------------------------ transfers
// Nested iso-interpolation (Sec. 3): weight 1 at coincident nodes, 1/2 at lateral or radial
// edge midpoints, 1/4 where both apply.  Lateral parents of fine lattice position (i, j):
// even/even -> (i/2, j/2); odd i -> ((i-1)/2, j/2), ((i+1)/2, j/2); odd j -> (i/2, (j-1)/2),
// (i/2, (j+1)/2); odd/odd -> midpoint of the coarse anti-diagonal ((i+1)/2, (j-1)/2), ((i-1)/2, (j+1)/2).
// Semi-coarsened level pairs (lateral factor lf or radial factor rf equal to 1) keep the
// index in that direction (weight 1).
template <typename T>
__global__ void k_prolong(Dims F, Dims C, int lf, int rf, int ncomp, int apply_bc, const T* __restrict__ c0,
                          const T* __restrict__ c1, const T* __restrict__ c2, T* f0, T* f1, T* f2,
                          const T* __restrict__ svec, int bc_in, int bc_out) {
  const int N = F.N, M = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: fine lattice points x F.n_r x 10
  if (t >= M * M) return;
  const int i = t / M, j = t - i * M, k = blockIdx.y, d = blockIdx.z;
  int li[2], lj[2], nl;
  if (lf == 1 || (!(i & 1) && !(j & 1))) {
    li[0] = lf == 1 ? i : i / 2, lj[0] = lf == 1 ? j : j / 2, nl = 1;
  } else if ((i & 1) && !(j & 1)) {
    li[0] = (i - 1) / 2, lj[0] = j / 2, li[1] = (i + 1) / 2, lj[1] = j / 2, nl = 2;
  } else if (!(i & 1) && (j & 1)) {
    li[0] = i / 2, lj[0] = (j - 1) / 2, li[1] = i / 2, lj[1] = (j + 1) / 2, nl = 2;
  } else {
    li[0] = (i + 1) / 2, lj[0] = (j - 1) / 2, li[1] = (i - 1) / 2, lj[1] = (j + 1) / 2, nl = 2;
  }
  int rk[2], nrk;
  if (rf == 1) rk[0] = k, nrk = 1;
  else if (!(k & 1)) rk[0] = k / 2, nrk = 1;
  else rk[0] = (k - 1) / 2, rk[1] = (k + 1) / 2, nrk = 2;
  const T* cs[3] = {c0, c1, c2};
  T* fs[3] = {f0, f1, f2};
  T v[3];
  for (int c = 0; c < ncomp; ++c) {
    T rad[2];
    for (int r = 0; r < nrk; ++r) {
      const int64_t b = (int64_t)d * C.diamond_stride + (int64_t)rk[r] * C.layer_stride;
      rad[r] = nl == 1 ? cs[c][b + (int64_t)li[0] * C.P + lj[0]]
                       : (T)0.5 * (cs[c][b + (int64_t)li[0] * C.P + lj[0]] + cs[c][b + (int64_t)li[1] * C.P + lj[1]]);
    }
    v[c] = nrk == 1 ? rad[0] : (T)0.5 * (rad[0] + rad[1]);
  }
  if (apply_bc && ncomp == 3 && (k == 0 || k == F.n_r - 1))
    project_vec(v, svec, ((int64_t)d * M + i) * F.P + j, F.n_lat_layout, k == 0 ? bc_in : bc_out);
  const int64_t idx = (int64_t)d * F.diamond_stride + (int64_t)k * F.layer_stride + (int64_t)i * F.P + j;
  for (int c = 0; c < ncomp; ++c) fs[c][idx] = v[c];
}

// Restriction P^T: coarse node (I, J, K) gathers the fine nodes it interpolates to (semi-coarsened
// pairs keep the index in the direction with factor 1): lateral
// (2I, 2J) with weight 1 and its six lattice neighbours with weight 1/2, radial 2K (1) and
// 2K +- 1 (1/2).  Fine nodes shared by several diamonds are counted by their canonical copy
// only; the coarse copies are then summed by launch_interface.
template <typename T>
__global__ void k_restrict(Dims F, Dims C, int lf, int rf, int ncomp, const uint8_t* __restrict__ owned,
                           const T* __restrict__ f0, const T* __restrict__ f1, const T* __restrict__ f2, T* c0, T* c1,
                           T* c2) {
  const int NC = C.N, MC = NC + 1, NF = F.N, MF = NF + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: coarse lattice points x C.n_r x 10
  if (t >= MC * MC) return;
  const int I = t / MC, J = t - I * MC, K = blockIdx.y, d = blockIdx.z;
  const int nb[7][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
  const T* fs[3] = {f0, f1, f2};
  T* cs[3] = {c0, c1, c2};
  T v[3] = {0, 0, 0};
  for (int r = -1; r <= 1; ++r) {
    if (rf == 1 && r != 0) continue;
    const int kf = rf * K + r;
    if (kf < 0 || kf >= F.n_r) continue;
    const T wr = r == 0 ? (T)1 : (T)0.5;
    T lat[3] = {0, 0, 0};
    for (int q = 0; q < (lf == 1 ? 1 : 7); ++q) {
      const int fi = lf * I + nb[q][0], fj = lf * J + nb[q][1];
      if (fi < 0 || fj < 0 || fi > NF || fj > NF) continue;
      if (!owned[((int64_t)d * MF + fi) * F.P + fj]) continue;
      const T wl = q == 0 ? (T)1 : (T)0.5;
      const int64_t idx = (int64_t)d * F.diamond_stride + (int64_t)kf * F.layer_stride + (int64_t)fi * F.P + fj;
      for (int c = 0; c < ncomp; ++c) lat[c] += wl * fs[c][idx];
    }
    for (int c = 0; c < ncomp; ++c) v[c] += wr * lat[c];
  }
  const int64_t idx = (int64_t)d * C.diamond_stride + (int64_t)K * C.layer_stride + (int64_t)I * C.P + J;
  for (int c = 0; c < ncomp; ++c) cs[c][idx] = v[c];
}

// In-place projection of the boundary layers (after a restriction's interface sum).
template <typename T>
__global__ void k_project_bdry(Dims D, T* y0, T* y1, T* y2, const T* __restrict__ svec, int bc_in, int bc_out) {
  const int M = D.N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: lattice points x 2 layers x 10 diamonds
  if (t >= M * M) return;
  const int i = t / M, j = t - i * M, side = blockIdx.y, d = blockIdx.z;
  const int k = side == 0 ? 0 : D.n_r - 1;
  const int64_t idx = (int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride + (int64_t)i * D.P + j;
  T v[3] = {y0[idx], y1[idx], y2[idx]};
  project_vec(v, svec, ((int64_t)d * M + i) * D.P + j, D.n_lat_layout, side == 0 ? bc_in : bc_out);
  y0[idx] = v[0], y1[idx] = v[1], y2[idx] = v[2];
}

// ------------------------------------------------------------------------------------ diag(M_1/eta)
// Thread per coarse (pressure) node: sum over the coarse wedges around it and their 8 fine
// children of V_e / eta_e psi_k(q_c^e)^2.  psi_k at a child's barycentre is the coarse W1
// basis at the child's barycentre in the coarse reference wedge: lateral (2/3, 1/6, 1/6)
// (permuted) for the three corner children, (1/3, 1/3, 1/3) for the middle one; radial
// (3/4, 1/4) for the lower child layer and (1/4, 3/4) for the upper one.
template <typename T>
__global__ void k_diag_pmass(Dims F, Dims C, const T* __restrict__ geoF, const T* __restrict__ layF,
                             EtaView<T> etaF, T* m) {
  const int NC = C.N, MC = NC + 1, NF = F.N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: coarse lattice points x C.n_r x 10
  if (t >= MC * MC) return;
  const int I = t / MC, J = t - I * MC, K = blockIdx.y, d = blockIdx.z;
  const int tri[6][4] = {{0, 0, 0, 0}, {-1, 0, 0, 1}, {-1, 0, 1, 2}, {0, -1, 0, 2}, {0, -1, 1, 1}, {-1, -1, 1, 0}};
  // children of coarse W0 / W1: (fine di, fine dj, fine wedge), barycentric weight of local node a
  const int kid[2][4][3] = {{{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{1, 1, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}}};
  T acc = 0;
  for (int q = 0; q < 6; ++q) {
    const int ci = I + tri[q][0], cj = J + tri[q][1], w = tri[q][2], a = tri[q][3];
    if (ci < 0 || cj < 0 || ci >= NC || cj >= NC) continue;
    for (int side = 0; side < 2; ++side) {  // node is bottom of coarse layer K (side 0) or top of K-1
      const int kc = side == 0 ? K : K - 1;
      if (kc < 0 || kc >= C.n_r - 1) continue;
      for (int c = 0; c < 4; ++c) {
        const T wl = c == 3 ? (T)(1.0 / 3.0) : (c == a ? (T)(2.0 / 3.0) : (T)(1.0 / 6.0));
        const int fi = 2 * ci + kid[w][c][0], fj = 2 * cj + kid[w][c][1], fw = kid[w][c][2];
        const int64_t t = (((int64_t)d * NF + fi) * NF + fj) * 2 + fw;
        const T dM = geoF[(int64_t)9 * F.n_tri + t];
        for (int r = 0; r < 2; ++r) {
          const int kf = 2 * kc + r;
          // weight of this coarse node: bottom node (side 0) -> 3/4 in lower child, 1/4 in upper
          const T wr = (side == 0) == (r == 0) ? (T)0.75 : (T)0.25;
          const T psi = wl * wr;
          const T V = layF[kLayerStride * kf + 2] * dM;
          const T e = eta_at(etaF, ((((int64_t)d * (F.n_r - 1) + kf) * NF + fi) * NF + fj) * 2 + fw, t);
          acc += V / e * psi * psi;
        }
      }
    }
  }
  m[(int64_t)d * C.diamond_stride + (int64_t)K * C.layer_stride + (int64_t)I * C.P + J] = acc;
}

// ------------------------------------------------------------------------------------ viscosity
// lay[kLayerStride k + 3] holds the layer mid-radius (r_k + r_k+1) / 2.
#if TN_PART == 0 || TN_PART == 1
__global__ void k_eta_from_T(Dims D, const double* __restrict__ T, double E, double jump_r, double jump_f,
                             const double* __restrict__ lay, double* eta) {
  const int N = D.N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: lateral wedges x (n_r - 1) x 10 diamonds
  if (t >= 2 * N * N) return;
  const int i = t / (2 * N), r = t - i * 2 * N, j = r >> 1, w = r & 1, k = blockIdx.y, d = blockIdx.z;
  const int64_t tid = (((int64_t)d * (D.n_r - 1) + k) * N * N + (int64_t)i * N + j) * 2 + w;  // wedge index
  int pi_[3], pj_[3];
  if (w == 0) pi_[0] = i, pj_[0] = j, pi_[1] = i + 1, pj_[1] = j, pi_[2] = i, pj_[2] = j + 1;
  else pi_[0] = i + 1, pj_[0] = j + 1, pi_[1] = i, pj_[1] = j + 1, pi_[2] = i + 1, pj_[2] = j;
  const int64_t b = (int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride;
  double s = 0;
  for (int a = 0; a < 3; ++a) s += T[b + (int64_t)pi_[a] * D.P + pj_[a]];
  for (int a = 0; a < 3; ++a) s += T[b + D.layer_stride + (int64_t)pi_[a] * D.P + pj_[a]];
  const double Te = s / 6.0;
  double e = exp(E * (0.5 - Te));
  if (jump_r > 0 && lay[kLayerStride * k + 3] < jump_r) e = jump_f * e;
  eta[tid] = e;
}

__global__ void k_eta_coarsen(Dims F, Dims C, int lf, int rf, const double* __restrict__ ef, double* ec) {
  const int NC = C.N, NF = F.N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: coarse lateral wedges x (C.n_r - 1) x 10
  if (t >= 2 * NC * NC) return;
  const int I = t / (2 * NC), r = t - I * 2 * NC, J = r >> 1, w = r & 1, K = blockIdx.y, d = blockIdx.z;
  const int64_t tid = (((int64_t)d * (C.n_r - 1) + K) * NC * NC + (int64_t)I * NC + J) * 2 + w;  // wedge index
  const int kid[2][4][3] = {{{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{1, 1, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}}};
  double s = 0;
  const int nlat = lf == 2 ? 4 : 1;
  for (int c = 0; c < nlat; ++c)
    for (int r = 0; r < rf; ++r) {
      const int fi = lf == 2 ? 2 * I + kid[w][c][0] : I, fj = lf == 2 ? 2 * J + kid[w][c][1] : J;
      const int fw = lf == 2 ? kid[w][c][2] : w, kf = rf * K + r;
      s += ef[((((int64_t)d * (F.n_r - 1) + kf) * NF + fi) * NF + fj) * 2 + fw];
    }
  ec[tid] = s / (double)(nlat * rf);
}

__global__ void k_to_f32(const double* __restrict__ a, float* b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------------------------ buoyancy
// f_j = sum_e V_e Ra T(q_c) r_hat(q_c) / 6 with r_hat(q_c) = sbar / |sbar| (x(q_c) = rho sbar).
// With a reference state (TALA, Eq. stokes) each radial cell's term carries cellw[k] =
// rho(q_c) alpha(q_c), and T is the perturbation T'.
__global__ void k_buoyancy(Dims D, const double* __restrict__ geo, const double* __restrict__ lay,
                           const double* __restrict__ svec, const double* __restrict__ T, double Ra, int bc_in,
                           int bc_out, const double* __restrict__ cellw, double* f0, double* f1, double* f2) {
  const int N = D.N, M = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // grid: lattice points x n_r x 10 diamonds
  if (t >= M * M) return;
  const int i = t / M, j = t - i * M, k = blockIdx.y, d = blockIdx.z;
  const int tri[6][4] = {{0, 0, 0, 0}, {-1, 0, 0, 1}, {-1, 0, 1, 2}, {0, -1, 0, 2}, {0, -1, 1, 1}, {-1, -1, 1, 0}};
  double f[3] = {0, 0, 0};
  for (int q = 0; q < 6; ++q) {
    const int ci = i + tri[q][0], cj = j + tri[q][1], w = tri[q][2];
    if (ci < 0 || cj < 0 || ci >= N || cj >= N) continue;
    int pi_[3], pj_[3];
    if (w == 0) pi_[0] = ci, pj_[0] = cj, pi_[1] = ci + 1, pj_[1] = cj, pi_[2] = ci, pj_[2] = cj + 1;
    else pi_[0] = ci + 1, pj_[0] = cj + 1, pi_[1] = ci, pj_[1] = cj + 1, pi_[2] = ci + 1, pj_[2] = cj;
    double sb[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) sb[c] += svec[((int64_t)d * M + pi_[a]) * D.P + pj_[a] + c * D.n_lat_layout];
    const double nrm = sqrt(sb[0] * sb[0] + sb[1] * sb[1] + sb[2] * sb[2]);
    const int64_t t = (((int64_t)d * N + ci) * N + cj) * 2 + w;
    const double dM = geo[(int64_t)9 * D.n_tri + t];
    for (int side = 0; side < 2; ++side) {
      const int kk = side == 0 ? k : k - 1;
      if (kk < 0 || kk >= D.n_r - 1) continue;
      const int64_t b = (int64_t)d * D.diamond_stride + (int64_t)kk * D.layer_stride;
      double s = 0;
      for (int a = 0; a < 3; ++a) s += T[b + (int64_t)pi_[a] * D.P + pj_[a]];
      for (int a = 0; a < 3; ++a) s += T[b + D.layer_stride + (int64_t)pi_[a] * D.P + pj_[a]];
      const double V = lay[kLayerStride * kk + 2] * dM;
      double wgt = V * Ra * (s / 6.0) / 6.0 / nrm;
      if (cellw) wgt *= cellw[kk];
      for (int c = 0; c < 3; ++c) f[c] += wgt * sb[c];
    }
  }
  const bool shared = i == 0 || i == N || j == 0 || j == N;
  (void)shared;
  if (k == 0 || k == D.n_r - 1)
    project_vec(f, svec, ((int64_t)d * M + i) * D.P + j, D.n_lat_layout, k == 0 ? bc_in : bc_out);
  const int64_t idx = (int64_t)d * D.diamond_stride + (int64_t)k * D.layer_stride + (int64_t)i * D.P + j;
  f0[idx] = f[0], f1[idx] = f[1], f2[idx] = f[2];
}

#endif  // TN_PART == 0 || TN_PART == 1

}  // namespace

// ---------------------------------------------------------------------------------------- launchers
// kappa (3 + c) / 18 of the hourglass control (c = 1/3 with the div term, 1 without).
inline double hg_coef(const Level& L, int div_term) {
  return L.hg_kappa * (3.0 + (div_term ? 1.0 / 3.0 : 1.0)) / 18.0;
}

// FP64 levels that run the halo-free tiles take the double-float element op when the mesh asks
// for it (tn_mesh_opts.fp64_element); every other level and precision the op of its own type.
template <typename T>
inline bool use_df(const Level& L) {
  return sizeof(T) == 8 && L.df && TN_WIDE_TILES && TN_HALO_FREE && L.N >= 2 * TILE;
}

// The FP32 A apply on paired-cell tiles (pair32.cuh) serves levels with N >= 32 whose three input
// arrays start on 16-byte boundaries; the others take the square tiles.
inline bool pair32_ok(const Level& L, const float* const* in) {
  auto al = [](const float* p) { return ((uintptr_t)p & 15) == 0; };
  return TN_PAIR32 && L.quad == 1 && L.N >= 2 * TILE && L.ring64 && L.grp_dij && L.n_layout < (int64_t)INT32_MAX &&
         L.n_wedges < (int64_t)INT32_MAX && al(in[0]) && al(in[1]) && al(in[2]);
}

template <bool HG, int EPI>
cudaError_t launch_pair32(const Level& L, BC bc, const OpA<float, HG>& op, const float* const* in, float* const* out,
                          cudaStream_t st, const int* skip, const EpiArgs<float>* epi) {
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  EpiArgs<float> E{};
  if (epi) E = *epi;
  const Dims D = dims(L);
  const int ntiles = (L.N / kPTI) * (L.N / kPTJ), ncells = L.n_r - 1;
  int kc = ncells;
  while (kc > kPMaxKc || (kc > TN_KC_MIN && (int64_t)ntiles * 10 * ((ncells + kc - 1) / kc) < TN_PAIR_CTA_TARGET))
    kc = (kc + 1) / 2;
  const dim3 grid(ntiles, (ncells + kc - 1) / kc, 10);
  const EtaView<float> ev = etav<float>(L);
  float4* const ring = reinterpret_cast<float4*>(L.ring64);  // 16 floats per 12 doubles of the FP64 layout
#define TN_PAIR_LAUNCH(EKv)                                                                                    \
  k_pair32<HG, F, EPI, EKv><<<grid, kPThreads, kPSmemBytes, st>>>(D, op, in[0], in[1], in[2], out[0], out[1],   \
                                                                 out[2], L.geo32, L.lay32, ev, L.s32, bc.in,     \
                                                                 bc.out, kc, skip, E, ring)
  if (ev.kind == TN_ETA_BF16) TN_PAIR_LAUNCH(TN_ETA_BF16);
  else if (ev.kind == TN_ETA_F16) TN_PAIR_LAUNCH(TN_ETA_F16);
  else TN_PAIR_LAUNCH(TN_ETA_F32);
#undef TN_PAIR_LAUNCH
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const RingDims RD = ring_dims(L.N, kPTI, kPTJ);
  k_ring4_fix<F, EPI><<<dim3(nblk(RD.RC, 256), L.n_r, 10), 256, 0, st>>>(D, RD, ring, in[0], in[1], in[2], out[0],
                                                                        out[1], out[2], L.s32, bc.in, bc.out, skip, E);
  e = cudaGetLastError();
  if (e != cudaSuccess || L.n_groups == 0) return e;
  k_ring4_edges<EPI><<<dim3(nblk(L.n_groups, 128), L.n_r), 128, 0, st>>>(
      D, RD, L.n_groups, L.grp_ptr, L.grp_off, L.grp_dij, L.grp_s32, ring, in[0], in[1], in[2], out[0], out[1], out[2],
      bc.in, bc.out, skip, E);
  return cudaGetLastError();
}

template <typename T, bool HG>
cudaError_t apply_A_hg(const Level& L, BC bc, int div_term, const T* const* u, T* const* y, cudaStream_t st,
                       const int* skip) {
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  if constexpr (sizeof(T) == 8) {
    if (use_df<T>(L)) {
      OpA<dfl, HG> op{div_term, dfl(hg_coef(L, div_term))};
      return launch_tile<T, OpA<dfl, HG>, F>(L, bc, op, u, y, etav<T>(L), st, skip);
    }
  }
  OpA<T, HG> op{div_term, (T)hg_coef(L, div_term)};
  return launch_tile<T, OpA<T, HG>, F>(L, bc, op, u, y, etav<T>(L), st, skip);
}

// The tile launches of the A apply with the second radial quadrature point (OpA2; their own
// translation units): plain, and with one of the fused epilogues.
template <typename T>
cudaError_t apply_A_q2(const Level& L, BC bc, int div_term, const T* const* u, T* const* y, cudaStream_t st,
                       const int* skip);
template <typename T>
cudaError_t apply_A_q2_epi(const Level& L, BC bc, int div_term, int epi, const T* const* in, const EpiArgs<T>& E,
                           T* const* t, cudaStream_t st, const int* skip);
// Shared-memory opt-ins of the OpA2 tile kernels (see prepare_tile_kernels).
cudaError_t prepare_tile_kernels_q2();
// Shared-memory opt-ins of the FP32 paired-cell A kernels (defined with their launchers).
cudaError_t prepare_tile_kernels_f32();

// The FP32 A apply on paired-cell tiles, interface sums included (pair32.cuh).
template <bool HG>
cudaError_t pair32_apply(const Level& L, BC bc, int div_term, int epi, const float* const* in, float* const* out,
                         cudaStream_t st, const int* skip, const EpiArgs<float>* E) {
  const OpA<float, HG> op{div_term, (float)hg_coef(L, div_term)};
  switch (epi) {
    case EPI_NONE: return launch_pair32<HG, EPI_NONE>(L, bc, op, in, out, st, skip, nullptr);
    case EPI_RESID: return launch_pair32<HG, EPI_RESID>(L, bc, op, in, out, st, skip, E);
    case EPI_CHEB1: return launch_pair32<HG, EPI_CHEB1>(L, bc, op, in, out, st, skip, E);
    case EPI_CHEB2: return launch_pair32<HG, EPI_CHEB2>(L, bc, op, in, out, st, skip, E);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_apply_A(const Level& L, BC bc, int div_term, const T* const* u, T* const* y, cudaStream_t st,
                           const int* skip) {
  if constexpr (sizeof(T) == 4) {
    if (pair32_ok(L, u))
      return L.hg_kappa > 0 ? pair32_apply<true>(L, bc, div_term, EPI_NONE, u, y, st, skip, nullptr)
                            : pair32_apply<false>(L, bc, div_term, EPI_NONE, u, y, st, skip, nullptr);
  }
  cudaError_t e = L.quad == 2      ? apply_A_q2<T>(L, bc, div_term, u, y, st, skip)
                  : L.hg_kappa > 0 ? apply_A_hg<T, true>(L, bc, div_term, u, y, st, skip)
                                   : apply_A_hg<T, false>(L, bc, div_term, u, y, st, skip);
  if (e != cudaSuccess) return e;
  return launch_interface<T>(L, bc, 3, 1, y, u, st, skip);
}

template <typename T, bool HG>
cudaError_t apply_A_epi_hg(const Level& L, BC bc, int div_term, int epi, const T* const* in, const EpiArgs<T>& E,
                           T* const* t, cudaStream_t st, const int* skip) {
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  if constexpr (sizeof(T) == 8) {
    if (use_df<T>(L)) {
      using Od = OpA<dfl, HG>;
      const Od od{div_term, dfl(hg_coef(L, div_term))};
      switch (epi) {
        case EPI_RESID: return launch_tile<T, Od, F, EPI_RESID>(L, bc, od, in, t, etav<T>(L), st, skip, &E);
        case EPI_CHEB1: return launch_tile<T, Od, F, EPI_CHEB1>(L, bc, od, in, t, etav<T>(L), st, skip, &E);
        case EPI_CHEB2: return launch_tile<T, Od, F, EPI_CHEB2>(L, bc, od, in, t, etav<T>(L), st, skip, &E);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  OpA<T, HG> op{div_term, (T)hg_coef(L, div_term)};
  using Op = OpA<T, HG>;
  switch (epi) {
    case EPI_RESID: return launch_tile<T, Op, F, EPI_RESID>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    case EPI_CHEB1: return launch_tile<T, Op, F, EPI_CHEB1>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    case EPI_CHEB2: return launch_tile<T, Op, F, EPI_CHEB2>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_apply_A_epi(const Level& L, BC bc, int div_term, int epi, const T* const* in, const EpiArgs<T>& E,
                               T* const* t, cudaStream_t st, const int* skip) {
  if constexpr (sizeof(T) == 4) {
    if (pair32_ok(L, in)) {
      if (epi != EPI_RESID && epi != EPI_CHEB1 && epi != EPI_CHEB2) return cudaErrorInvalidValue;
      return L.hg_kappa > 0 ? pair32_apply<true>(L, bc, div_term, epi, in, t, st, skip, &E)
                            : pair32_apply<false>(L, bc, div_term, epi, in, t, st, skip, &E);
    }
  }
  cudaError_t e = L.quad == 2      ? apply_A_q2_epi<T>(L, bc, div_term, epi, in, E, t, st, skip)
                  : L.hg_kappa > 0 ? apply_A_epi_hg<T, true>(L, bc, div_term, epi, in, E, t, st, skip)
                                   : apply_A_epi_hg<T, false>(L, bc, div_term, epi, in, E, t, st, skip);
  if (e != cudaSuccess) return e;
  const int64_t n = (int64_t)L.n_groups * L.n_r;
  if (n == 0) return cudaSuccess;
  const dim3 nb(nblk(L.n_groups, 128), L.n_r);
  const Dims D = dims(L);
#define TN_IEPI(EP)                                                                                             \
  k_interface_epi<T, EP><<<nb, 128, 0, st>>>(D, L.n_groups, L.grp_ptr, L.grp_off, Tab<T>::gs(L), t[0], t[1], t[2], \
                                             in[0], in[1], in[2], bc.in, bc.out, skip, E)
  if (epi == EPI_RESID) TN_IEPI(EPI_RESID);
  else if (epi == EPI_CHEB1) TN_IEPI(EPI_CHEB1);
  else TN_IEPI(EPI_CHEB2);
#undef TN_IEPI
  return cudaGetLastError();
}

#if TN_PART == 0 || TN_PART == 1
template <typename T>
cudaError_t launch_div_fine(const Level& L, BC bc, const T* const* u, T* q, cudaStream_t st) {
  T* out[1] = {q};
  cudaError_t e = cudaSuccess;
  bool done = false;
  const int nt = (int)L.n_tri;
  if constexpr (sizeof(T) == 8) {
    if (use_df<T>(L)) {
      const dfl* rh = reinterpret_cast<const dfl*>(L.rhatdf);
      e = L.tala ? launch_tile<T, OpDiv<dfl, true>, PROJ_IN>(L, bc, OpDiv<dfl, true>{rh, nt}, u, out, EtaView<T>{}, st)
                 : launch_tile<T, OpDiv<dfl>, PROJ_IN>(L, bc, OpDiv<dfl>{}, u, out, EtaView<T>{}, st);
      done = true;
    }
  }
  if (!done) {
    const T* rh = sizeof(T) == 8 ? (const T*)L.rhat64 : (const T*)L.rhat32;
    e = L.tala ? launch_tile<T, OpDiv<T, true>, PROJ_IN>(L, bc, OpDiv<T, true>{rh, nt}, u, out, EtaView<T>{}, st)
               : launch_tile<T, OpDiv<T>, PROJ_IN>(L, bc, OpDiv<T>{}, u, out, EtaView<T>{}, st);
  }
  if (e != cudaSuccess) return e;
  return launch_interface<T>(L, bc, 1, 0, out, nullptr, st);
}

template <typename T>
cudaError_t launch_grad_fine(const Level& L, BC bc, const T* p, T* const* y, cudaStream_t st) {
  const T* in[1] = {p};
  cudaError_t e = cudaSuccess;
  bool done = false;
  if constexpr (sizeof(T) == 8) {
    if (use_df<T>(L)) {
      e = launch_tile<T, OpGrad<dfl>, PROJ_OUT>(L, bc, OpGrad<dfl>{}, in, y, EtaView<T>{}, st);
      done = true;
    }
  }
  if (!done) e = launch_tile<T, OpGrad<T>, PROJ_OUT>(L, bc, OpGrad<T>{}, in, y, EtaView<T>{}, st);
  if (e != cudaSuccess) return e;
  return launch_interface<T>(L, bc, 3, 0, y, nullptr, st);
}

template <typename T>
cudaError_t launch_diag_A(const Level& L, BC bc, int div_term, T* const* d, cudaStream_t st) {
  Dims D = dims(L);
  // interior layers: per-cell tile kernel (boundary layers are overwritten below)
  const T* none[1] = {d[0]};
  const T hgk = (T)hg_coef(L, div_term);
  const bool hg = L.hg_kappa > 0;
  cudaError_t e;
  if (L.quad == 2) {  // second radial quadrature point: gradient form, both precisions
    e = launch_tile<T, OpDiag2<T>, 0>(L, bc, OpDiag2<T>{div_term}, none, d, etav<T>(L), st);
  } else if constexpr (sizeof(T) == 8) {  // FP64: per-triangle factor table
    if (!L.dcoef64 || L.dcoef_div != div_term) return cudaErrorInvalidValue;  // built with the level
    const int nt = (int)L.n_tri;
    if (use_df<T>(L)) {  // the table's double-float copy
      if (!L.dcoefdf) return cudaErrorInvalidValue;
      const dfl* cdf = reinterpret_cast<const dfl*>(L.dcoefdf);
      const dfl hk(hg_coef(L, div_term));
      if (!hg && !L.dcoefdf2) return cudaErrorInvalidValue;
      e = hg ? launch_tile<T, OpDiag<dfl, true>, 0>(L, bc, OpDiag<dfl, true>{div_term, hk, cdf, nt}, none, d,
                                                    etav<T>(L), st)
             : launch_tile<T, OpDiag<dfl, false>, 0>(L, bc, OpDiag<dfl, false>{div_term, hk, L.dcoefdf2, nt / 2},
                                                     none, d, etav<T>(L), st);
    } else {
      const T* coef = Tab<T>::dcoef(L);
      e = hg ? launch_tile<T, OpDiag<T, true>, 0>(L, bc, OpDiag<T, true>{div_term, hgk, coef, nt}, none, d,
                                                 etav<T>(L), st)
             : launch_tile<T, OpDiag<T, false>, 0>(L, bc, OpDiag<T, false>{div_term, hgk, coef, nt}, none, d,
                                                  etav<T>(L), st);
    }
  } else {  // FP32: gradient form
    e = hg ? launch_tile<T, OpDiagG<T, true>, 0>(L, bc, OpDiagG<T, true>{div_term, hgk}, none, d, etav<T>(L), st)
           : launch_tile<T, OpDiagG<T, false>, 0>(L, bc, OpDiagG<T, false>{div_term, hgk}, none, d, etav<T>(L), st);
  }
  if (e != cudaSuccess) return e;
  k_diag_A<T><<<dim3(nblk((int64_t)(L.N + 1) * (L.N + 1), 256), 2, 10), 256, 0, st>>>(D, Tab<T>::geo(L), Tab<T>::lay(L), etav<T>(L), Tab<T>::s(L), bc.in,
                                            bc.out, div_term, hgk, L.quad, d[0], d[1], d[2]);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_interface<T>(L, bc, 3, 2, d, nullptr, st);
}

template <typename T>
cudaError_t launch_block_inv_A(const Level& L, BC bc, int div_term, T* const* b, cudaStream_t st) {
  Dims D = dims(L);
  k_block_A<T><<<dim3(nblk((int64_t)(L.N + 1) * (L.N + 1), 256), L.n_r, 10), 256, 0, st>>>(D, Tab<T>::geo(L), Tab<T>::lay(L), etav<T>(L), Tab<T>::s(L), bc.in,
                                             bc.out, div_term, (T)hg_coef(L, div_term), L.quad, b[0], b[1], b[2], b[3],
                                             b[4],
                                             b[5]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ng = (int64_t)L.n_groups * L.n_r;
  if (ng > 0) {
    k_interface_block<T><<<nblk(ng, 128), 128, 0, st>>>(D, L.n_groups, L.grp_ptr, L.grp_off, Tab<T>::gs(L), b[0], b[1],
                                                        b[2], b[3], b[4], b[5], bc.in, bc.out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_block_inv<T><<<nblk(L.n_layout, 256), 256, 0, st>>>(L.n_layout, b[0], b[1], b[2], b[3], b[4], b[5]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag_pmass(const Level& F, const Level& C, T* m, cudaStream_t st) {
  k_diag_pmass<T><<<dim3(nblk((int64_t)(C.N + 1) * (C.N + 1), 256), C.n_r, 10), 256, 0, st>>>(dims(F), dims(C), Tab<T>::geo(F), Tab<T>::lay(F), etav<T>(F), m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  T* out[1] = {m};
  return launch_interface<T>(C, BC{0, 0}, 1, 0, out, nullptr, st);
}

template <typename T>
cudaError_t launch_interface(const Level& L, BC bc, int ncomp, int mode, T* const* y, const T* const* u,
                             cudaStream_t st, const int* skip) {
  const int64_t n = (int64_t)L.n_groups * L.n_r;
  if (n == 0) return cudaSuccess;
  T* y1 = ncomp > 1 ? y[1] : y[0];
  T* y2 = ncomp > 2 ? y[2] : y[0];
  const T* u0 = u ? u[0] : nullptr;
  const T* u1 = u ? u[1] : nullptr;
  const T* u2 = u ? u[2] : nullptr;
  k_interface<T><<<dim3(nblk(L.n_groups, 128), L.n_r), 128, 0, st>>>(dims(L), L.n_groups, L.grp_ptr, L.grp_off,
                                                                   Tab<T>::gs(L), ncomp, mode,
                                               y[0], y1, y2, u0, u1, u2, bc.in, bc.out, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const Level& F, const Level& C, BC bc, int ncomp, int apply_bc, const T* const* c,
                           T* const* f, cudaStream_t st) {
  const T* c1 = ncomp > 1 ? c[1] : c[0];
  const T* c2 = ncomp > 2 ? c[2] : c[0];
  T* f1 = ncomp > 1 ? f[1] : f[0];
  T* f2 = ncomp > 2 ? f[2] : f[0];
  const int lf = F.N / C.N, rf = (F.n_r - 1) / (C.n_r - 1);
  k_prolong<T><<<dim3(nblk((int64_t)(F.N + 1) * (F.N + 1), 256), F.n_r, 10), 256, 0, st>>>(dims(F), dims(C), lf, rf, ncomp, apply_bc, c[0], c1, c2, f[0], f1, f2,
                                             Tab<T>::s(F), bc.in, bc.out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Level& F, const Level& C, BC bc, int ncomp, int apply_bc, const T* const* f,
                            T* const* c, cudaStream_t st) {
  const T* f1 = ncomp > 1 ? f[1] : f[0];
  const T* f2 = ncomp > 2 ? f[2] : f[0];
  T* c1 = ncomp > 1 ? c[1] : c[0];
  T* c2 = ncomp > 2 ? c[2] : c[0];
  const int lf = F.N / C.N, rf = (F.n_r - 1) / (C.n_r - 1);
  k_restrict<T><<<dim3(nblk((int64_t)(C.N + 1) * (C.N + 1), 256), C.n_r, 10), 256, 0, st>>>(dims(F), dims(C), lf, rf, ncomp, F.owned, f[0], f1, f2, c[0], c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_interface<T>(C, bc, ncomp, 0, c, nullptr, st);
  if (e != cudaSuccess || !(apply_bc && ncomp == 3)) return e;
  k_project_bdry<T><<<dim3(nblk((int64_t)(C.N + 1) * (C.N + 1), 256), 2, 10), 256, 0, st>>>(dims(C), c[0], c[1], c[2], Tab<T>::s(C), bc.in, bc.out);
  return cudaGetLastError();
}

cudaError_t launch_eta_from_T(const Level& L, const double* T, double E, double jump_r, double jump_f, double* eta,
                              cudaStream_t st) {
  k_eta_from_T<<<dim3(nblk((int64_t)2 * L.N * L.N, 256), L.n_r - 1, 10), 256, 0, st>>>(dims(L), T, E, jump_r, jump_f, L.lay64, eta);
  return cudaGetLastError();
}

cudaError_t launch_eta_coarsen(const Level& F, const Level& C, const double* ef, double* ec, cudaStream_t st) {
  const int lf = F.N / C.N, rf = (F.n_r - 1) / (C.n_r - 1);
  k_eta_coarsen<<<dim3(nblk((int64_t)2 * C.N * C.N, 256), C.n_r - 1, 10), 256, 0, st>>>(dims(F), dims(C), lf, rf, ef, ec);
  return cudaGetLastError();
}

// Thread per lateral wedge column t = ((d N + i) N + j) 2 + w: c = sqrt(min * max) of the FP64
// viscosity over the column's n_r - 1 cells (rounded to FP32), then each value stored as the
// 16-bit rounding (to nearest even) of the FP32 rounding of eta / c.
template <int KIND>
__global__ void k_eta_16(Dims D, const double* __restrict__ eta, uint16_t* __restrict__ q, float* __restrict__ cs) {
  const int64_t per_d = (int64_t)2 * D.N * D.N;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 10 * per_d) return;
  const int64_t base = (t / per_d) * (D.n_r - 1) * per_d + t % per_d;  // wedge index at k = 0
  double mn = eta[base], mx = eta[base];
  for (int k = 1; k < D.n_r - 1; ++k) {
    const double e = eta[base + k * per_d];
    mn = fmin(mn, e), mx = fmax(mx, e);
  }
  const float c = (float)sqrt(mn * mx);
  cs[t] = c;
  for (int k = 0; k < D.n_r - 1; ++k) {
    const float r = (float)(eta[base + k * per_d] / (double)c);
    q[base + k * per_d] = KIND == TN_ETA_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(r))
                                              : __half_as_ushort(__float2half_rn(r));
  }
}

int64_t ring_buffer_entries(int N, int n_r) {
  if (!(TN_HALO_FREE && N >= 2 * TILE)) return 0;
  const RingDims RD = ring_dims(N, TILE, 2 * TILE);
  return (int64_t)4 * 3 * n_r * 10 * RD.RC;
}

cudaError_t launch_eta_f32_path(const Level& L, cudaStream_t st) {
  if (L.eta_kind == TN_ETA_F32) return launch_to_f32(L.eta64, L.eta32, L.n_wedges, st);
  if (L.eta_kind == TN_ETA_BF16)
    k_eta_16<TN_ETA_BF16><<<nblk(L.n_tri, 256), 256, 0, st>>>(dims(L), L.eta64, L.eta16, L.eta_cs);
  else
    k_eta_16<TN_ETA_F16><<<nblk(L.n_tri, 256), 256, 0, st>>>(dims(L), L.eta64, L.eta16, L.eta_cs);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t st) {
  k_to_f32<<<nblk(n, 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_buoyancy(const Level& L, BC bc, const double* T, double Ra, double* const* f, cudaStream_t st) {
  k_buoyancy<<<dim3(nblk((int64_t)(L.N + 1) * (L.N + 1), 256), L.n_r, 10), 256, 0, st>>>(dims(L), L.geo64, L.lay64, L.s64, T, Ra, bc.in, bc.out, L.bw64, f[0],
                                           f[1], f[2]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_interface<double>(L, bc, 3, 0, f, nullptr, st);
}

#define TN_INST(T)                                                                                               \
  template cudaError_t launch_div_fine<T>(const Level&, BC, const T* const*, T*, cudaStream_t);                 \
  template cudaError_t launch_grad_fine<T>(const Level&, BC, const T*, T* const*, cudaStream_t);                \
  template cudaError_t launch_diag_A<T>(const Level&, BC, int, T* const*, cudaStream_t);                        \
  template cudaError_t launch_block_inv_A<T>(const Level&, BC, int, T* const*, cudaStream_t);                   \
  template cudaError_t launch_diag_pmass<T>(const Level&, const Level&, T*, cudaStream_t);                      \
  template cudaError_t launch_interface<T>(const Level&, BC, int, int, T* const*, const T* const*, cudaStream_t,  \
                                           const int*);                                                          \
  template cudaError_t launch_prolong<T>(const Level&, const Level&, BC, int, int, const T* const*, T* const*,   \
                                         cudaStream_t);                                                         \
  template cudaError_t launch_restrict<T>(const Level&, const Level&, BC, int, int, const T* const*, T* const*,  \
                                          cudaStream_t);
TN_INST(double)
TN_INST(float)
#undef TN_INST
#endif  // TN_PART == 0 || TN_PART == 1

#define TN_INST_A(T)                                                                                             \
  template cudaError_t launch_apply_A<T>(const Level&, BC, int, const T* const*, T* const*, cudaStream_t,       \
                                         const int*);                                                            \
  template cudaError_t launch_apply_A_epi<T>(const Level&, BC, int, int, const T* const*, const EpiArgs<T>&,     \
                                             T* const*, cudaStream_t, const int*);
// Opt the tile kernels that need more than 48 KB of shared memory (FP64 A on 16 x 32 tiles,
// every epilogue, each A op) into their dynamic size.
template <typename Op, int EPI>
cudaError_t set_wide_a_attr() {
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  constexpr size_t sh = TileSmem<double, Op, TILE, 2 * TILE>::bytes;
  if (sh > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_wide<double, Op, TILE, 2 * TILE, F, EPI, TN_ETA_F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  constexpr size_t shf = TileSmemHF<double, Op, TILE, 2 * TILE>::bytes;
  if (shf > 48 * 1024)
    return cudaFuncSetAttribute(k_tile_hf<double, Op, TILE, 2 * TILE, F, EPI, TN_ETA_F32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf);
  return cudaSuccess;
}

template <typename Op>
cudaError_t set_wide_attrs() {
  const cudaError_t e[4] = {set_wide_a_attr<Op, EPI_NONE>(), set_wide_a_attr<Op, EPI_RESID>(),
                            set_wide_a_attr<Op, EPI_CHEB1>(), set_wide_a_attr<Op, EPI_CHEB2>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

// The double-float A ops (halo-free tiles only).
template <typename Op, int EPI>
cudaError_t set_df_attr() {
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  constexpr size_t shf = TileSmemHF<dfl, Op, TILE, 2 * TILE>::bytes;
  if (shf > 48 * 1024)
    return cudaFuncSetAttribute(k_tile_hf<double, Op, TILE, 2 * TILE, F, EPI, TN_ETA_F32, dfl>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf);
  return cudaSuccess;
}
template <typename Op>
cudaError_t set_df_attrs() {
  const cudaError_t e[4] = {set_df_attr<Op, EPI_NONE>(), set_df_attr<Op, EPI_RESID>(), set_df_attr<Op, EPI_CHEB1>(),
                            set_df_attr<Op, EPI_CHEB2>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

#if TN_PART == 0 || TN_PART == 2
TN_INST_A(double)

// Energy residual (Eq. energy) and lumped mass on level L, FP64: R = (K + C(u) + S(u)) T with the
// element op OpEnergy (u NULL: diffusion only), plus the interface sum over diamond-edge copies.
// Defined in this part, beside the shared-memory opt-in of its tile kernel.
cudaError_t launch_energy_residual(const Level& L, const double* const* u, const double* T, double* R, int supg,
                                   cudaStream_t st) {
  const double* in[4] = {u ? u[0] : T, u ? u[1] : T, u ? u[2] : T, T};
  double* out[1] = {R};
  const BC bc{TN_BC_FREESLIP, TN_BC_FREESLIP};  // no projection flags: the boundary conditions do not enter R
  cudaError_t e = launch_tile<double, OpEnergy<double>, 0>(L, bc, OpEnergy<double>{u ? 1 : 0, supg}, in, out,
                                                           EtaView<double>{}, st);
  if (e != cudaSuccess) return e;
  return launch_interface<double>(L, bc, 1, 0, out, nullptr, st);
}

cudaError_t launch_lumped_mass(const Level& L, double* m, cudaStream_t st) {
  const double* none[1] = {m};
  double* out[1] = {m};
  const BC bc{TN_BC_FREESLIP, TN_BC_FREESLIP};
  cudaError_t e = launch_tile<double, OpMass<double>, 0>(L, bc, OpMass<double>{}, none, out, EtaView<double>{}, st);
  if (e != cudaSuccess) return e;
  return launch_interface<double>(L, bc, 1, 0, out, nullptr, st);
}

cudaError_t prepare_energy_kernels() {
  constexpr size_t sh = TileSmemHF<double, OpEnergy<double>, TILE, 2 * TILE>::bytes;
  if (sh > 48 * 1024)
    return cudaFuncSetAttribute(k_tile_hf<double, OpEnergy<double>, TILE, 2 * TILE, 0, EPI_NONE, TN_ETA_F32, double>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  return cudaSuccess;
}

cudaError_t prepare_tile_kernels() {
  const cudaError_t e[7] = {prepare_tile_kernels_f32(), set_wide_attrs<OpA<double, false>>(), set_wide_attrs<OpA<double, true>>(),
                            set_df_attrs<OpA<dfl, false>>(), set_df_attrs<OpA<dfl, true>>(),
                            prepare_tile_kernels_q2(), prepare_energy_kernels()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
#endif
#if TN_PART == 0 || TN_PART == 3
TN_INST_A(float)
template <bool HG, int EPI, int EK>
cudaError_t set_pair32_attr() {
  return cudaFuncSetAttribute(k_pair32<HG, PROJ_IN | PROJ_OUT | ADD_ID, EPI, EK>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmemBytes);
}
template <bool HG, int EPI>
cudaError_t set_pair32_attrs() {
  const cudaError_t e[3] = {set_pair32_attr<HG, EPI, TN_ETA_F32>(), set_pair32_attr<HG, EPI, TN_ETA_BF16>(),
                            set_pair32_attr<HG, EPI, TN_ETA_F16>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
cudaError_t prepare_tile_kernels_f32() {
  const cudaError_t e[8] = {set_pair32_attrs<false, EPI_NONE>(), set_pair32_attrs<false, EPI_RESID>(),
                            set_pair32_attrs<false, EPI_CHEB1>(), set_pair32_attrs<false, EPI_CHEB2>(),
                            set_pair32_attrs<true, EPI_NONE>(),  set_pair32_attrs<true, EPI_RESID>(),
                            set_pair32_attrs<true, EPI_CHEB1>(),  set_pair32_attrs<true, EPI_CHEB2>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}
#endif
#undef TN_INST_A

// ------------------------------------------------------------ A with the second radial point
// Defined in parts 4 and 5 only: the other parts link to these instantiations (an implicit one
// elsewhere would launch that part's own copy of the tile kernels, without the shared-memory
// opt-in of prepare_tile_kernels_q2).
#if TN_PART == 0 || TN_PART == 4 || TN_PART == 5
template <typename T>
cudaError_t apply_A_q2(const Level& L, BC bc, int div_term, const T* const* u, T* const* y, cudaStream_t st,
                       const int* skip) {
  return launch_tile<T, OpA2<T>, PROJ_IN | PROJ_OUT | ADD_ID>(L, bc, OpA2<T>{div_term}, u, y, etav<T>(L), st, skip);
}

template <typename T>
cudaError_t apply_A_q2_epi(const Level& L, BC bc, int div_term, int epi, const T* const* in, const EpiArgs<T>& E,
                           T* const* t, cudaStream_t st, const int* skip) {
  using Op = OpA2<T>;
  const Op op{div_term};
  constexpr int F = PROJ_IN | PROJ_OUT | ADD_ID;
  switch (epi) {
    case EPI_RESID: return launch_tile<T, Op, F, EPI_RESID>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    case EPI_CHEB1: return launch_tile<T, Op, F, EPI_CHEB1>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    case EPI_CHEB2: return launch_tile<T, Op, F, EPI_CHEB2>(L, bc, op, in, t, etav<T>(L), st, skip, &E);
    default: return cudaErrorInvalidValue;
  }
}

#endif

#define TN_INST_Q2(T)                                                                                            \
  template cudaError_t apply_A_q2<T>(const Level&, BC, int, const T* const*, T* const*, cudaStream_t, const int*); \
  template cudaError_t apply_A_q2_epi<T>(const Level&, BC, int, int, const T* const*, const EpiArgs<T>&,         \
                                         T* const*, cudaStream_t, const int*);
#if TN_PART == 0 || TN_PART == 4
TN_INST_Q2(double)
cudaError_t prepare_tile_kernels_q2() { return set_wide_attrs<OpA2<double>>(); }
#endif
#if TN_PART == 0 || TN_PART == 5
TN_INST_Q2(float)
#endif
#undef TN_INST_Q2

}  // namespace tn
