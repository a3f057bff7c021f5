// Solver layer: deterministic reductions, Chebyshev / geometric-multigrid V-cycle and the
// FGMRES Stokes solve with the block-triangular preconditioner (Sec. 7, Eq. block-precond,
// Eq. pmass), in FP64 or as FP32 inner solves inside FP64 iterative refinement.
//
// Orchestration is host C++ enqueueing kernels on one stream.  Inner products always
// accumulate in FP64 over unique nodes (the canonical copy of every diamond-edge node) and
// reduce in a fixed order, so every result is bitwise reproducible.  The coarsest-level
// conjugate-gradient loop keeps its scalars on the device and stops through a device flag
// (later kernels of a converged loop return immediately), so a V-cycle needs no host sync.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace tn {

namespace {

constexpr int RG = 304;   // blocks of a reduction (fixed: the summation order never changes)
constexpr int RB = 256;   // threads per reduction block
constexpr int MAXV = 12;  // vectors per multi-dot / multi-axpy
constexpr int EB = 256;   // elementwise block size

inline unsigned nb(int64_t n) { return (unsigned)((n + EB - 1) / EB); }

template <typename T>
struct Ptr4 {
  const T* c[4];
};
template <typename T>
struct MPtr4 {
  T* c[4];
};
template <typename T>
struct B6 {  // inverse 3x3 node blocks (xx, yy, zz, xy, xz, yz)
  const T* c[6];
};
template <typename T>
__device__ __forceinline__ void bmul(const B6<T>& b, int64_t i, const T (&r)[3], T (&z)[3]) {
  const T a = b.c[0][i], e = b.c[1][i], f = b.c[2][i], xy = b.c[3][i], xz = b.c[4][i], yz = b.c[5][i];
  z[0] = a * r[0] + xy * r[1] + xz * r[2];
  z[1] = xy * r[0] + e * r[1] + yz * r[2];
  z[2] = xz * r[0] + yz * r[1] + f * r[2];
}
template <typename T>
struct DotArgs {
  const T* x[MAXV][4];
  const T* y[4];
};
template <typename T>
struct AxpyArgs {
  const T* x[MAXV][4];
  T* y[4];
};

// ------------------------------------------------------------------------------------- reductions
// part[v * RG + block] = sum over masked entries of sum_c x[v][c] y[c]
template <typename T>
__global__ void __launch_bounds__(RB) k_dots(int64_t n, const uint8_t* __restrict__ mask, int nvec, int ncomp,
                                             DotArgs<T> a, double* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip) return;
  // FP64 accumulators; products are formed in T and, for FP32 vectors, summed in FP32 over
  // at most 8 consecutive elements of a thread before they are added in FP64.
  double acc[MAXV];
  T pacc[MAXV];
#pragma unroll
  for (int v = 0; v < MAXV; ++v) acc[v] = 0.0, pacc[v] = (T)0;
  int cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)RG * RB) {
    if (!mask[i]) continue;
    T yv[4];
    for (int c = 0; c < ncomp; ++c) yv[c] = a.y[c][i];
#pragma unroll
    for (int v = 0; v < MAXV; ++v) {
      if (v < nvec) {
        T s = (T)0;
        for (int c = 0; c < ncomp; ++c) s += a.x[v][c][i] * yv[c];
        if (sizeof(T) == 8) acc[v] += (double)s;
        else pacc[v] += s;
      }
    }
    if (sizeof(T) != 8 && ++cnt == 8) {
#pragma unroll
      for (int v = 0; v < MAXV; ++v) acc[v] += (double)pacc[v], pacc[v] = (T)0;
      cnt = 0;
    }
  }
  if (sizeof(T) != 8) {
#pragma unroll
    for (int v = 0; v < MAXV; ++v) acc[v] += (double)pacc[v];
  }
  __shared__ double sh[RB / 32][MAXV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < MAXV; ++v) {
    if (v < nvec) {
      double s = acc[v];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) sh[wid][v] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double s = 0.0;
    for (int w = 0; w < RB / 32; ++w) s += sh[w][threadIdx.x];
    part[threadIdx.x * RG + blockIdx.x] = s;
  }
}

// out[v] = sum_b part0[v RG + b] (+ part1[v RG + b]) in a fixed order; block per vector.
__global__ void k_dots_final(int nvec, const double* __restrict__ part0, const double* __restrict__ part1,
                             double* __restrict__ out, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int v = blockIdx.x;
  __shared__ double sh[RB];
  double s = 0.0;
  for (int b = threadIdx.x; b < RG; b += RB) {
    double t = part0[v * RG + b];
    if (part1) t += part1[v * RG + b];
    s += t;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = sh[0];
}

// Angular momentum sum over unique nodes of x cross u (three dots with the rigid rotations
// e_i x x, since <u, e_i x x> = e_i . (x cross u)).
template <typename T>
__global__ void __launch_bounds__(RB) k_angmom(Dims D, const uint8_t* __restrict__ mask, const T* __restrict__ svec,
                                               const T* __restrict__ rad, Ptr4<T> u, double* __restrict__ part,
                                               const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t n = 10 * D.diamond_stride;
  double acc[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)RG * RB) {
    if (!mask[i]) continue;
    const int64_t d = i / D.diamond_stride, rem = i % D.diamond_stride;
    const int k = (int)(rem / D.layer_stride);
    const int64_t lat = d * (int64_t)(D.N + 1) * D.P + rem % D.layer_stride;
    const double r = rad[k];
    const double x[3] = {r * svec[lat], r * svec[lat + D.n_lat_layout], r * svec[lat + 2 * D.n_lat_layout]};
    const double w[3] = {u.c[0][i], u.c[1][i], u.c[2][i]};
    acc[0] += x[1] * w[2] - x[2] * w[1];
    acc[1] += x[2] * w[0] - x[0] * w[2];
    acc[2] += x[0] * w[1] - x[1] * w[0];
  }
  __shared__ double sh[RB / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = 0; v < 3; ++v) {
    double s = acc[v];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[wid][v] = s;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < RB / 32; ++w) s += sh[w][threadIdx.x];
    part[threadIdx.x * RG + blockIdx.x] = s;
  }
}

// u -= (Ginv L) x x at every layout entry (L = angular momentum in Lm[0..2]).
struct M33 {
  double a[3][3];
};
template <typename T>
__global__ void k_sub_rotation(Dims D, const T* __restrict__ svec, const T* __restrict__ rad, MPtr4<T> u,
                               const double* __restrict__ Lm, M33 Ginv, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  const int64_t n = 10 * D.diamond_stride;
  if (i >= n) return;
  const int64_t d = i / D.diamond_stride, rem = i % D.diamond_stride;
  const int j = (int)(rem % D.P);
  if (j > D.N) return;
  const int k = (int)(rem / D.layer_stride);
  const int64_t lat = d * (int64_t)(D.N + 1) * D.P + rem % D.layer_stride;
  double w[3];
  for (int a = 0; a < 3; ++a) w[a] = Ginv.a[a][0] * Lm[0] + Ginv.a[a][1] * Lm[1] + Ginv.a[a][2] * Lm[2];
  const double r = rad[k];
  const double x[3] = {r * svec[lat], r * svec[lat + D.n_lat_layout], r * svec[lat + 2 * D.n_lat_layout]};
  u.c[0][i] -= (T)(w[1] * x[2] - w[2] * x[1]);
  u.c[1][i] -= (T)(w[2] * x[0] - w[0] * x[2]);
  u.c[2][i] -= (T)(w[0] * x[1] - w[1] * x[0]);
}

// --------------------------------------------------------------------------------- elementwise
// y[c] += sign * sum_v coef[v] x[v][c]  (coef on the device)
template <typename T>
__global__ void k_axpy_multi(int64_t n, int nvec, int ncomp, const double* __restrict__ coef, double sign,
                             AxpyArgs<T> a, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  T cf[MAXV];
  for (int v = 0; v < nvec; ++v) cf[v] = (T)(sign * coef[v]);
  for (int c = 0; c < ncomp; ++c) {
    T s = a.y[c][i];
    for (int v = 0; v < nvec; ++v) s += cf[v] * a.x[v][c][i];
    a.y[c][i] = s;
  }
}

// y[c] = alpha x[c] + beta y[c] with host scalars
template <typename T>
__global__ void k_axpby(int64_t n, int ncomp, double alpha, Ptr4<T> x, double beta, MPtr4<T> y) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T a = (T)alpha, b = (T)beta;
  for (int c = 0; c < ncomp; ++c) {
    const T xv = alpha != 0.0 ? a * x.c[c][i] : (T)0;
    const T yv = beta != 0.0 ? b * y.c[c][i] : (T)0;
    y.c[c][i] = xv + yv;
  }
}

// y[c] = x[c] * s, s = sqrt(1 / S[0]) (unit-normalise by a device squared norm)
template <typename T>
__global__ void k_normalize(int64_t n, int ncomp, Ptr4<T> x, MPtr4<T> y, const double* __restrict__ nrm2) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T s = (T)(1.0 / sqrt(nrm2[0]));
  for (int c = 0; c < ncomp; ++c) y.c[c][i] = x.c[c][i] * s;
}

// y = Binv x (block Jacobi)
template <typename T>
__global__ void k_bmul(int64_t n, B6<T> binv, Ptr4<T> x, MPtr4<T> y) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T r[3] = {x.c[0][i], x.c[1][i], x.c[2][i]};
  T z[3];
  bmul(binv, i, r, z);
  for (int c = 0; c < 3; ++c) y.c[c][i] = z[c];
}

template <typename T>
__global__ void k_recip(int64_t n, const T* __restrict__ d, T* __restrict__ inv) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T v = d[i];
  inv[i] = v != (T)0 ? (T)1 / v : (T)0;
}

// Chebyshev step, part 1 (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1, with the
// block-Jacobi preconditioner D^-1 = inverse 3x3 node blocks):
// r = b - t (t = K x; zero_x: x = 0, t unused), d = D^-1 r / theta, x += d
template <typename T>
__global__ void k_cheb1(int64_t n, int zero_x, double inv_theta, Ptr4<T> b, Ptr4<T> t, B6<T> binv, MPtr4<T> r,
                        MPtr4<T> d, MPtr4<T> x) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  T rr[3], z[3];
  for (int c = 0; c < 3; ++c) rr[c] = zero_x ? b.c[c][i] : b.c[c][i] - t.c[c][i];
  bmul(binv, i, rr, z);
  for (int c = 0; c < 3; ++c) {
    const T dd = (T)inv_theta * z[c];
    r.c[c][i] = rr[c];
    d.c[c][i] = dd;
    x.c[c][i] = zero_x ? dd : x.c[c][i] + dd;
  }
}
// part 2: r -= t (t = K d), d = c1 d + c2 D^-1 r, x += d
template <typename T>
__global__ void k_cheb2(int64_t n, double c1, double c2, Ptr4<T> t, B6<T> binv, MPtr4<T> r, MPtr4<T> d,
                        MPtr4<T> x) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  T rr[3], z[3];
  for (int c = 0; c < 3; ++c) rr[c] = r.c[c][i] - t.c[c][i];
  bmul(binv, i, rr, z);
  for (int c = 0; c < 3; ++c) {
    const T dd = (T)c1 * d.c[c][i] + (T)c2 * z[c];
    r.c[c][i] = rr[c];
    d.c[c][i] = dd;
    x.c[c][i] = x.c[c][i] + dd;
  }
}

// ---- coarse CG (device scalars in S, stop flag) ----------------------------------------------
constexpr int MAX_RESTART = 30;
enum { S_RZ0 = 0, S_RZ = 1, S_PQ = 2, S_RZN = 3, S_ALPHA = 4, S_BETA = 5, S_QR = 6, S_TMP = 8, S_L = 12, S_H = 16,
       S_H2 = S_H + MAX_RESTART + 1, S_NRM = S_H2 + MAX_RESTART + 1, S_Y = S_NRM + 1, S_MAX = S_Y + MAX_RESTART + 1 };

__global__ void k_cg_alpha(double* S, const int* __restrict__ skip) {
  if (skip && *skip) return;
  S[S_ALPHA] = S[S_RZ] / S[S_PQ];
}
// x += alpha p; r -= alpha q; z = D^-1 r
template <typename T>
__global__ void k_cg_update(int64_t n, const double* __restrict__ S, Ptr4<T> p, Ptr4<T> q, B6<T> binv, MPtr4<T> x,
                            MPtr4<T> r, MPtr4<T> z, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T al = (T)S[S_ALPHA];
  T rr[3], zz[3];
  for (int c = 0; c < 3; ++c) {
    x.c[c][i] += al * p.c[c][i];
    rr[c] = r.c[c][i] - al * q.c[c][i];
    r.c[c][i] = rr[c];
  }
  bmul(binv, i, rr, zz);
  for (int c = 0; c < 3; ++c) z.c[c][i] = zz[c];
}
__global__ void k_cg_beta(double* S, int* flag, double tol2, int last) {
  if (*flag) return;
  S[S_BETA] = S[S_RZN] / S[S_RZ];
  S[S_RZ] = S[S_RZN];
  if (!(S[S_RZN] > tol2 * S[S_RZ0]) || last) *flag = 1;
}
template <typename T>
__global__ void k_cg_dir(int64_t n, const double* __restrict__ S, Ptr4<T> z, MPtr4<T> p, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T be = (T)S[S_BETA];
  for (int c = 0; c < 3; ++c) p.c[c][i] = z.c[c][i] + be * p.c[c][i];
}
// Coarse CG on a small coarsest level (n <= SMALL_CG): one block runs the whole vector part of a
// CG step, so a step is the operator apply plus one launch.  Sums over the masked (unique)
// entries in FP64, in a fixed order (thread-strided partial sums, then a tree over the block).
constexpr int SMALL_CG = 32768;
constexpr int SB = 1024;  // threads of the single-block CG kernels

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // sh may still be read from a previous sum
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < SB / 32; ++w) s += sh[w];  // every thread, same order
  return s;
}

// r = b, z = D^-1 r, p = z, x = 0, rz0 = (r, z); flag = 0 unless rz0 = 0
template <typename T>
__global__ void __launch_bounds__(SB) k_cg_start_small(int64_t n, const uint8_t* __restrict__ mask, Ptr4<T> b,
                                                       B6<T> binv, MPtr4<T> r, MPtr4<T> z, MPtr4<T> p, MPtr4<T> x,
                                                       double* S, int* flag) {
  __shared__ double sh[SB / 32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += SB) {
    T rr[3] = {b.c[0][i], b.c[1][i], b.c[2][i]}, zz[3];
    bmul(binv, i, rr, zz);
    T d = (T)0;
    for (int c = 0; c < 3; ++c) {
      r.c[c][i] = rr[c], z.c[c][i] = zz[c], p.c[c][i] = zz[c], x.c[c][i] = (T)0;
      d += rr[c] * zz[c];
    }
    if (mask[i]) acc += (double)d;
  }
  const double rz0 = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    S[S_RZ0] = rz0, S[S_RZ] = rz0;
    *flag = rz0 > 0.0 ? 0 : 1;
  }
}

// one CG step after q = K p: alpha = (r, z) / (p, q); x += alpha p; r -= alpha q; z = D^-1 r;
// beta = (r, z)_new / (r, z); p = z + beta p; flag once (r, z) <= tol2 (r0, z0) or at the last step
template <typename T>
__global__ void __launch_bounds__(SB) k_cg_step_small(int64_t n, const uint8_t* __restrict__ mask, MPtr4<T> p,
                                                      Ptr4<T> q, B6<T> binv, MPtr4<T> x, MPtr4<T> r, MPtr4<T> z,
                                                      double* S, int* flag, double tol2, int last) {
  if (*flag) return;
  __shared__ double sh[SB / 32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += SB) {
    if (!mask[i]) continue;
    T d = (T)0;
    for (int c = 0; c < 3; ++c) d += p.c[c][i] * q.c[c][i];
    acc += (double)d;
  }
  const double pq = block_sum(acc, sh);
  const double rz = S[S_RZ];
  const T al = (T)(rz / pq);
  acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += SB) {
    T rr[3], zz[3];
    for (int c = 0; c < 3; ++c) {
      x.c[c][i] += al * p.c[c][i];
      rr[c] = r.c[c][i] - al * q.c[c][i];
      r.c[c][i] = rr[c];
    }
    bmul(binv, i, rr, zz);
    T d = (T)0;
    for (int c = 0; c < 3; ++c) z.c[c][i] = zz[c], d += rr[c] * zz[c];
    if (mask[i]) acc += (double)d;
  }
  const double rzn = block_sum(acc, sh);
  const bool stop = !(rzn > tol2 * S[S_RZ0]) || last;
  if (!stop) {
    const T be = (T)(rzn / rz);
    for (int64_t i = threadIdx.x; i < n; i += SB)
      for (int c = 0; c < 3; ++c) p.c[c][i] = z.c[c][i] + be * p.c[c][i];
  }
  __syncthreads();  // every thread has read S[S_RZ] and S[S_RZ0]
  if (threadIdx.x == 0) {
    S[S_RZ] = rzn;
    if (stop) *flag = 1;
  }
}

__global__ void k_set_int(int* f, int v) { *f = v; }
__global__ void k_cg_start(double* S, int* flag) {
  S[S_RZ] = S[S_RZ0];
  *flag = S[S_RZ0] > 0.0 ? 0 : 1;
}

template <typename T, typename U>
__global__ void k_convert(int64_t n, const T* __restrict__ a, U* __restrict__ b, double scale) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i < n) b[i] = (U)((double)a[i] * scale);
}
// x64 += scale * d32
template <typename T>
__global__ void k_accum(int64_t n, const T* __restrict__ d, double* __restrict__ x, double scale) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i < n) x[i] += scale * (double)d[i];
}
// z_p = -r_p / m (m = diag(M_1/eta); 0 on padding)
template <typename T>
__global__ void k_schur(int64_t n, const T* __restrict__ m, const T* __restrict__ r, T* __restrict__ z) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T mm = m[i];
  z[i] = mm != (T)0 ? -r[i] / mm : (T)0;
}

// Deflated Schur step (DEF2 with the constant vector q, Tang, Nabben, Vuik, Erlangga 2009):
// t = q^T r / q^T S q, z = -(r - S q t) / m + q t; q = 1, S q precomputed.
template <typename T>
__global__ void k_schur_defl(int64_t n, const T* __restrict__ m, const T* __restrict__ r, const T* __restrict__ sq,
                             const double* __restrict__ qr, double inv_qsq, T* __restrict__ z) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i >= n) return;
  const T mm = m[i];
  const T t = (T)(qr[0] * inv_qsq);
  z[i] = mm != (T)0 ? -(r[i] - sq[i] * t) / mm + t : (T)0;
}
template <typename T>
__global__ void k_fill(int64_t n, T v, T* __restrict__ a) {
  const int64_t i = blockIdx.x * (int64_t)EB + threadIdx.x;
  if (i < n) a[i] = v;
}

// SplitMix64 (Steele, Lea, Flood 2014) -> uniform in [-1, 1)
inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

// ============================================================================ multigrid state
template <typename T>
struct Vec3 {
  T* c[3] = {nullptr, nullptr, nullptr};
  const T* const* cc() const { return (const T* const*)c; }
  T* const* mm() const { return (T* const*)c; }
};

template <typename T>
struct MGLevelT {
  // x and d are double-buffered: the fused Chebyshev updates write the new x (or d) while the
  // apply still reads the old one; xi / di select the current buffer.
  Vec3<T> xb[2], b, r, db[2], t, p;  // p only on the coarsest level
  int xi = 0, di = 0;
  Vec3<T>& x() { return xb[xi]; }
  Vec3<T>& d() { return db[di]; }
  T* binv[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // inverse node blocks
  double lam = 0.0;
  B6<T> bi() const {
    B6<T> b;
    for (int q = 0; q < 6; ++q) b.c[q] = binv[q];
    return b;
  }
};

template <typename T>
struct KVec {  // composite (u on level 0, p on level 1)
  T* u[3] = {nullptr, nullptr, nullptr};
  T* p = nullptr;
};

template <typename T>
struct PrecState {
  bool ready = false;
  std::vector<MGLevelT<T>> L;
  T* mdiag = nullptr;                 // diag(M_1/eta) on level 1
  T* ones_p = nullptr;                // 1 on every pressure layout entry (level 1)
  T* sq = nullptr;                    // S 1 ~ -B A^-1 P B^T 1 (deflation of the constant pressure mode)
  double qsq = 0.0;                   // 1^T S 1 over unique pressure nodes (0: deflation off)
  Vec3<T> defl_w, defl_c;             // A^-1 c and c = P B^T 1 (set-up work vectors)
  std::vector<KVec<T>> V, Z;          // FGMRES bases
  KVec<T> w, tmp;                     // work vectors
  KVec<T> ir_r, ir_c;                 // FP32 iterative refinement: inner rhs and correction
  cudaGraphExec_t vgraph = nullptr;   // the V-cycle (level-0 b -> level-0 x) captured after set-up
  cudaGraph_t vtemplate = nullptr;    // its graph, kept for composing several systems' V-cycles
  T* tu[3] = {nullptr, nullptr, nullptr};  // velocity scratch (level 0)
};

struct MGState {
  tn_mg_opts opts;
  int nlev = 0;
  // Multigrid levels: geo[0] is the mesh's level 0; coarser levels are owned here and may be
  // semi-coarsened (lateral only or radial only) where the cells are anisotropic.
  std::vector<Level*> geo;
  std::vector<Level*> owned_levels;
  double* S = nullptr;     // device scalars
  int* flag = nullptr;     // coarse CG stop flag
  double* part = nullptr;  // reduction partials [2][MAXV][RG]
  PrecState<double> p64;
  PrecState<float> p32;
  std::vector<void*> allocs;
  int restart = 0;         // FGMRES bases allocated for this restart length
  cudaStream_t cap = nullptr;  // stream used to capture the V-cycle graphs
};

namespace {

template <typename T>
PrecState<T>& ps(MGState* m);
template <>
PrecState<double>& ps<double>(MGState* m) {
  return m->p64;
}
template <>
PrecState<float>& ps<float>(MGState* m) {
  return m->p32;
}
template <typename T>
const T* svec_of(const Level& L);
template <>
const double* svec_of<double>(const Level& L) {
  return L.s64;
}
template <>
const float* svec_of<float>(const Level& L) {
  return L.s32;
}
template <typename T>
const T* rad_of(const Level& L);
template <>
const double* rad_of<double>(const Level& L) {
  return L.rad64;
}
template <>
const float* rad_of<float>(const Level& L) {
  return L.rad32;
}

thread_local cudaError_t g_err = cudaSuccess;
inline void ck(cudaError_t e) {
  if (g_err == cudaSuccess && e != cudaSuccess) g_err = e;
}
inline void ckl() { ck(cudaGetLastError()); }

template <typename T>
T* alloc_zero(MGState* m, int64_t n) {
  void* p = nullptr;
  ck(cudaMalloc(&p, sizeof(T) * (size_t)n));
  if (p) {
    ck(cudaMemset(p, 0, sizeof(T) * (size_t)n));
    m->allocs.push_back(p);
  }
  return (T*)p;
}

template <typename T>
Vec3<T> alloc3(MGState* m, int64_t n) {
  Vec3<T> v;
  for (int c = 0; c < 3; ++c) v.c[c] = alloc_zero<T>(m, n);
  return v;
}

template <typename T>
Ptr4<T> P4(const T* const* c, int n) {
  Ptr4<T> p{};
  for (int i = 0; i < 4; ++i) p.c[i] = i < n ? c[i] : nullptr;
  return p;
}
template <typename T>
MPtr4<T> M4(T* const* c, int n) {
  MPtr4<T> p{};
  for (int i = 0; i < 4; ++i) p.c[i] = i < n ? c[i] : nullptr;
  return p;
}

// out[0..nvec) = dots of x[v] with y over unique nodes of level L (ncomp components).
template <typename T>
void dots(MGState* m, const Level& L, int nvec, int ncomp, const T* const* const* x, const T* const* y, double* out,
          cudaStream_t st, const int* skip = nullptr) {
  DotArgs<T> a{};
  for (int v = 0; v < nvec; ++v)
    for (int c = 0; c < ncomp; ++c) a.x[v][c] = x[v][c];
  for (int c = 0; c < ncomp; ++c) a.y[c] = y[c];
  k_dots<T><<<RG, RB, 0, st>>>(L.n_layout, L.wmask, nvec, ncomp, a, m->part, skip);
  ckl();
  k_dots_final<<<nvec, RB, 0, st>>>(nvec, m->part, nullptr, out, skip);
  ckl();
}

// composite dots: velocity part on level 0 plus pressure part on level 1 (chunks of MAXV vectors)
template <typename T>
void kdots(MGState* m, const tn_mesh* mesh, int nvec, const KVec<T>* const* x, const KVec<T>& y, double* out,
           cudaStream_t st) {
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  for (int v0 = 0; v0 < nvec; v0 += MAXV) {
    const int nv = std::min(MAXV, nvec - v0);
    DotArgs<T> a{};
    for (int v = 0; v < nv; ++v)
      for (int c = 0; c < 3; ++c) a.x[v][c] = x[v0 + v]->u[c];
    for (int c = 0; c < 3; ++c) a.y[c] = y.u[c];
    k_dots<T><<<RG, RB, 0, st>>>(L0.n_layout, L0.wmask, nv, 3, a, m->part, nullptr);
    ckl();
    DotArgs<T> b{};
    for (int v = 0; v < nv; ++v) b.x[v][0] = x[v0 + v]->p;
    b.y[0] = y.p;
    k_dots<T><<<RG, RB, 0, st>>>(L1.n_layout, L1.wmask, nv, 1, b, m->part + MAXV * RG, nullptr);
    ckl();
    k_dots_final<<<nv, RB, 0, st>>>(nv, m->part, m->part + MAXV * RG, out + v0, nullptr);
    ckl();
  }
}

template <typename T>
void kaxpy(const tn_mesh* mesh, int nvec, const KVec<T>* const* x, const double* coef, double sign, KVec<T>& y,
           cudaStream_t st) {
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  for (int v0 = 0; v0 < nvec; v0 += MAXV) {
    const int nv = std::min(MAXV, nvec - v0);
    AxpyArgs<T> a{};
    for (int v = 0; v < nv; ++v)
      for (int c = 0; c < 3; ++c) a.x[v][c] = x[v0 + v]->u[c];
    for (int c = 0; c < 3; ++c) a.y[c] = y.u[c];
    k_axpy_multi<T><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, nv, 3, coef + v0, sign, a, nullptr);
    ckl();
    AxpyArgs<T> b{};
    for (int v = 0; v < nv; ++v) b.x[v][0] = x[v0 + v]->p;
    b.y[0] = y.p;
    k_axpy_multi<T><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, nv, 1, coef + v0, sign, b, nullptr);
    ckl();
  }
}

template <typename T>
void kaxpby(const tn_mesh* mesh, double alpha, const KVec<T>& x, double beta, KVec<T>& y, cudaStream_t st) {
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  k_axpby<T><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, 3, alpha, P4<T>(x.u, 3), beta, M4<T>(y.u, 3));
  ckl();
  const T* xp[1] = {x.p};
  T* yp[1] = {y.p};
  k_axpby<T><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, 1, alpha, P4<T>(xp, 1), beta, M4<T>(yp, 1));
  ckl();
}

bool rotations_singular(const tn_mesh* mesh) {
  return mesh->bc_in == TN_BC_FREESLIP && mesh->bc_out == TN_BC_FREESLIP;
}

M33 inverse33(const double (&a)[3][3]) {
  M33 r{};
  double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1], c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2],
         c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
  r.a[0][0] = c00 / det;
  r.a[1][0] = c01 / det;
  r.a[2][0] = c02 / det;
  r.a[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
  r.a[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
  r.a[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
  r.a[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
  r.a[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
  r.a[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
  return r;
}

// u <- u - (rigid-rotation component of u), Euclidean over unique nodes of level L
template <typename T>
void project_rotations(MGState* m, const Level& L, T* const* u, cudaStream_t st, const int* skip = nullptr) {
  k_angmom<T><<<RG, RB, 0, st>>>(dims(L), L.wmask, svec_of<T>(L), rad_of<T>(L), P4<T>((const T* const*)u, 3),
                                 m->part, skip);
  ckl();
  k_dots_final<<<3, RB, 0, st>>>(3, m->part, nullptr, m->S + S_L, skip);
  ckl();
  k_sub_rotation<T><<<nb(L.n_layout), EB, 0, st>>>(dims(L), svec_of<T>(L), rad_of<T>(L), M4<T>(u, 3), m->S + S_L,
                                                   inverse33(L.inertia), skip);
  ckl();
}

template <typename T>
void apply_K_level(const tn_mesh* mesh, int h, const T* const* x, T* const* y, cudaStream_t st,
                   const int* skip = nullptr) {
  ck(launch_apply_A<T>(*mesh->mg->geo[h], BC{mesh->bc_in, mesh->bc_out}, mesh->div_term, x, y, st, skip));
}

// Block-Jacobi-preconditioned CG on the coarsest level: x = K^-1 b (x0 = 0); stops when
// (r, D^-1 r) <= rtol^2 (r0, D^-1 r0) or after max_iters.
template <typename T>
void coarse_cg(MGState* m, const tn_mesh* mesh, int h, cudaStream_t st) {
  MGLevelT<T>& C = ps<T>(m).L[h];
  const Level& L = *m->geo[h];
  const int64_t n = L.n_layout;
  const bool proj = rotations_singular(mesh);
  if (proj) project_rotations<T>(m, L, C.b.mm(), st);
  const double tol2s = m->opts.coarse_rtol * m->opts.coarse_rtol;
  if (n <= SMALL_CG) {  // single-block vector kernels: two launches per CG step plus the apply
    k_cg_start_small<T><<<1, SB, 0, st>>>(n, L.wmask, P4<T>(C.b.cc(), 3), C.bi(), M4<T>(C.r.mm(), 3),
                                          M4<T>(C.d().mm(), 3), M4<T>(C.p.mm(), 3), M4<T>(C.x().mm(), 3), m->S,
                                          m->flag);
    ckl();
    const int maxit = m->opts.coarse_max_iters;
    for (int it = 0; it < maxit; ++it) {
      apply_K_level<T>(mesh, h, C.p.cc(), C.t.mm(), st, m->flag);
      k_cg_step_small<T><<<1, SB, 0, st>>>(n, L.wmask, M4<T>(C.p.mm(), 3), P4<T>(C.t.cc(), 3), C.bi(),
                                           M4<T>(C.x().mm(), 3), M4<T>(C.r.mm(), 3), M4<T>(C.d().mm(), 3), m->S,
                                           m->flag, tol2s, it == maxit - 1);
      ckl();
    }
    if (proj) project_rotations<T>(m, L, C.x().mm(), st);
    return;
  }
  // r = b, z = D^-1 r (stored in d), p = z, x = 0
  k_axpby<T><<<nb(n), EB, 0, st>>>(n, 3, 1.0, P4<T>(C.b.cc(), 3), 0.0, M4<T>(C.r.mm(), 3));
  ckl();
  k_bmul<T><<<nb(n), EB, 0, st>>>(n, C.bi(), P4<T>(C.r.cc(), 3), M4<T>(C.d().mm(), 3));
  ckl();
  k_axpby<T><<<nb(n), EB, 0, st>>>(n, 3, 1.0, P4<T>(C.d().cc(), 3), 0.0, M4<T>(C.p.mm(), 3));
  ckl();
  k_axpby<T><<<nb(n), EB, 0, st>>>(n, 3, 0.0, P4<T>(C.d().cc(), 3), 0.0, M4<T>(C.x().mm(), 3));
  ckl();
  k_set_int<<<1, 1, 0, st>>>(m->flag, 0);
  ckl();
  const T* const* rr[1] = {C.r.cc()};
  dots<T>(m, L, 1, 3, rr, C.d().cc(), m->S + S_RZ0, st);
  k_cg_start<<<1, 1, 0, st>>>(m->S, m->flag);
  ckl();
  const double tol2 = m->opts.coarse_rtol * m->opts.coarse_rtol;
  const int maxit = m->opts.coarse_max_iters;
  for (int it = 0; it < maxit; ++it) {
    apply_K_level<T>(mesh, h, C.p.cc(), C.t.mm(), st, m->flag);
    const T* const* pp[1] = {C.p.cc()};
    dots<T>(m, L, 1, 3, pp, C.t.cc(), m->S + S_PQ, st, m->flag);
    k_cg_alpha<<<1, 1, 0, st>>>(m->S, m->flag);
    ckl();
    k_cg_update<T><<<nb(n), EB, 0, st>>>(n, m->S, P4<T>(C.p.cc(), 3), P4<T>(C.t.cc(), 3), C.bi(),
                                         M4<T>(C.x().mm(), 3), M4<T>(C.r.mm(), 3), M4<T>(C.d().mm(), 3), m->flag);
    ckl();
    dots<T>(m, L, 1, 3, rr, C.d().cc(), m->S + S_RZN, st, m->flag);
    k_cg_beta<<<1, 1, 0, st>>>(m->S, m->flag, tol2, it == maxit - 1);
    ckl();
    k_cg_dir<T><<<nb(n), EB, 0, st>>>(n, m->S, P4<T>(C.d().cc(), 3), M4<T>(C.p.mm(), 3), m->flag);
    ckl();
  }
  if (proj) project_rotations<T>(m, L, C.x().mm(), st);
}

// One degree-2 Chebyshev smoothing step on level h (rhs b): the two operator applications carry
// the vector updates in their epilogues (r = b - K x, d = D^-1 r / theta, x += d; then
// r -= K d, d = c1 d + c2 D^-1 r, x += d).
template <typename T>
EpiArgs<T> epi_of(MGLevelT<T>& G) {
  EpiArgs<T> E{};
  for (int c = 0; c < 3; ++c) E.b[c] = G.b.c[c], E.r[c] = G.r.c[c];
  for (int q = 0; q < 6; ++q) E.binv[q] = G.binv[q];
  return E;
}

template <typename T>
void cheb_step(MGState* m, const tn_mesh* mesh, int h, bool zero_x, cudaStream_t st) {
  MGLevelT<T>& G = ps<T>(m).L[h];
  const Level& L = *m->geo[h];
  const BC bc{mesh->bc_in, mesh->bc_out};
  const int64_t n = L.n_layout;
  const double a = m->opts.cheb_lo * G.lam, b = m->opts.cheb_hi * G.lam;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  const double rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
  if (zero_x) {
    k_cheb1<T><<<nb(n), EB, 0, st>>>(n, 1, 1.0 / theta, P4<T>(G.b.cc(), 3), P4<T>(G.b.cc(), 3), G.bi(),
                                     M4<T>(G.r.mm(), 3), M4<T>(G.d().mm(), 3), M4<T>(G.x().mm(), 3));
    ckl();
  } else {
    EpiArgs<T> E = epi_of(G);
    E.c0 = 1.0 / theta;
    for (int c = 0; c < 3; ++c) E.dout[c] = G.d().c[c], E.xout[c] = G.xb[1 - G.xi].c[c];
    ck(launch_apply_A_epi<T>(L, bc, mesh->div_term, EPI_CHEB1, G.x().cc(), E, G.t.mm(), st));
    G.xi = 1 - G.xi;
  }
  EpiArgs<T> E = epi_of(G);
  E.c1 = rho1 * rho0;
  E.c2 = 2.0 * rho1 / delta;
  for (int c = 0; c < 3; ++c) E.xacc[c] = G.x().c[c], E.xout[c] = G.x().c[c], E.dout[c] = G.db[1 - G.di].c[c];
  ck(launch_apply_A_epi<T>(L, bc, mesh->div_term, EPI_CHEB2, G.d().cc(), E, G.t.mm(), st));
  G.di = 1 - G.di;
}

// V-cycle on level h: x_h = V(b_h)
template <typename T>
void vcycle_level(MGState* m, const tn_mesh* mesh, int h, cudaStream_t st) {
  if (h == m->nlev - 1) {
    coarse_cg<T>(m, mesh, h, st);
    return;
  }
  MGLevelT<T>& G = ps<T>(m).L[h];
  MGLevelT<T>& C = ps<T>(m).L[h + 1];
  const Level& F = *m->geo[h];
  const Level& Lc = *m->geo[h + 1];
  const BC bc{mesh->bc_in, mesh->bc_out};
  const int64_t n = F.n_layout;
  // The cycle starts from x = 0, so the buffer choice is reset: every cycle (captured or not)
  // then leaves x in the same buffer and readers after it see the right one.
  G.xi = 0, G.di = 0;
  for (int s = 0; s < m->opts.pre_smooth; ++s) cheb_step<T>(m, mesh, h, s == 0, st);
  if (m->opts.pre_smooth == 0)
    k_axpby<T><<<nb(n), EB, 0, st>>>(n, 3, 0.0, P4<T>(G.b.cc(), 3), 0.0, M4<T>(G.x().mm(), 3)), ckl();
  // r = b - K x (fused into the apply)
  {
    EpiArgs<T> E = epi_of(G);
    ck(launch_apply_A_epi<T>(F, bc, mesh->div_term, EPI_RESID, G.x().cc(), E, G.t.mm(), st));
  }
  ck(launch_restrict<T>(F, Lc, bc, 3, 1, G.r.cc(), C.b.mm(), st));
  vcycle_level<T>(m, mesh, h + 1, st);
  ck(launch_prolong<T>(F, Lc, bc, 3, 1, C.x().cc(), G.t.mm(), st));
  k_axpby<T><<<nb(n), EB, 0, st>>>(n, 3, 1.0, P4<T>(G.t.cc(), 3), 1.0, M4<T>(G.x().mm(), 3));
  ckl();
  for (int s = 0; s < m->opts.post_smooth; ++s) cheb_step<T>(m, mesh, h, false, st);
}

double host_scalar(MGState* m, int slot, cudaStream_t st) {
  double v = 0;
  ck(cudaMemcpyAsync(&v, m->S + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  return v;
}

// One V-cycle on level 0 (G.b -> G.x of level 0) on stream st: the captured graph if there is
// one, else the kernels directly.
template <typename T>
void run_vcycle(MGState* m, const tn_mesh* mesh, cudaStream_t st) {
  PrecState<T>& P = ps<T>(m);
  if (P.vgraph) ck(cudaGraphLaunch(P.vgraph, st));
  else vcycle_level<T>(m, mesh, 0, st);
}

// Capture the V-cycle into a graph (kernel parameters such as the Chebyshev coefficients are
// fixed at capture, so this runs at the end of every set-up).
template <typename T>
void capture_vcycle(MGState* m, const tn_mesh* mesh) {
  PrecState<T>& P = ps<T>(m);
  if (P.vgraph) {
    cudaGraphExecDestroy(P.vgraph);
    P.vgraph = nullptr;
  }
  if (P.vtemplate) {
    cudaGraphDestroy(P.vtemplate);
    P.vtemplate = nullptr;
  }
  if (!m->cap) ck(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
  if (g_err != cudaSuccess) return;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return;
  vcycle_level<T>(m, mesh, 0, m->cap);
  cudaError_t e = cudaStreamEndCapture(m->cap, &g);
  if (e == cudaSuccess && g_err == cudaSuccess) {
    if (cudaGraphInstantiate(&P.vgraph, g, 0) != cudaSuccess) P.vgraph = nullptr;
  }
  if (P.vgraph) P.vtemplate = g;
  else if (g) cudaGraphDestroy(g);
  cudaGetLastError();
}

template <typename T>
tn_status mg_setup_t(tn_mesh* mesh, const void* const* v0, cudaStream_t st) {
  MGState* m = mesh->mg;
  PrecState<T>& P = ps<T>(m);
  const BC bc{mesh->bc_in, mesh->bc_out};
  if (P.L.empty()) {
    P.L.resize(m->nlev);
    for (int h = 0; h < m->nlev; ++h) {
      const int64_t n = m->geo[h]->n_layout;
      MGLevelT<T>& G = P.L[h];
      G.xb[0] = alloc3<T>(m, n), G.xb[1] = alloc3<T>(m, n), G.b = alloc3<T>(m, n), G.r = alloc3<T>(m, n);
      G.db[0] = alloc3<T>(m, n), G.db[1] = alloc3<T>(m, n);
      G.t = alloc3<T>(m, n);
      for (int q = 0; q < 6; ++q) G.binv[q] = alloc_zero<T>(m, n);
      if (h == m->nlev - 1) G.p = alloc3<T>(m, n);
    }
    P.mdiag = alloc_zero<T>(m, mesh->lv[1].n_layout);
    P.ones_p = alloc_zero<T>(m, mesh->lv[1].n_layout);
    P.sq = alloc_zero<T>(m, mesh->lv[1].n_layout);
    P.defl_w = alloc3<T>(m, mesh->lv[0].n_layout);
    P.defl_c = alloc3<T>(m, mesh->lv[0].n_layout);
  }
  if (g_err != cudaSuccess) return TN_ENOMEM;
  // block-Jacobi: inverse 3x3 node blocks of P A P + I - P on every level
  for (int h = 0; h < m->nlev; ++h) ck(launch_block_inv_A<T>(*m->geo[h], bc, mesh->div_term, P.L[h].binv, st));
  ck(launch_diag_pmass<T>(mesh->lv[0], mesh->lv[1], P.mdiag, st));
  // power-iteration start vectors: level 0 given or SplitMix64, coarser levels restricted
  {
    const Level& L = mesh->lv[0];
    MGLevelT<T>& G = P.L[0];
    if (v0) {
      for (int c = 0; c < 3; ++c)
        ck(cudaMemcpyAsync(G.x().c[c], v0[c], sizeof(T) * L.n_layout, cudaMemcpyDeviceToDevice, st));
    } else {
      std::vector<int64_t> canon((size_t)L.n_layout);
      tn_mesh_canonical_index(mesh, 0, canon.data());
      std::vector<T> hv((size_t)L.n_layout);
      for (int c = 0; c < 3; ++c) {
        for (int64_t i = 0; i < L.n_layout; ++i) {
          if (canon[i] < 0) {
            hv[i] = 0;
            continue;
          }
          uint64_t z = splitmix64(m->opts.seed ^ splitmix64((uint64_t)canon[i] * 3 + c));
          hv[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
        }
        ck(cudaMemcpyAsync(G.x().c[c], hv.data(), sizeof(T) * L.n_layout, cudaMemcpyHostToDevice, st));
        ck(cudaStreamSynchronize(st));
      }
    }
  }
  for (int h = 1; h < m->nlev; ++h)
    ck(launch_restrict<T>(*m->geo[h - 1], *m->geo[h], bc, 3, 1, P.L[h - 1].x().cc(), P.L[h].x().mm(), st));
  // power iterations on D^-1 K of every smoothing level
  std::vector<double> lam(m->nlev, 0.0);
  for (int h = 0; h + 1 < m->nlev; ++h) {
    MGLevelT<T>& G = P.L[h];
    const Level& L = *m->geo[h];
    const int64_t n = L.n_layout;
    const T* const* xx[1] = {G.x().cc()};
    dots<T>(m, L, 1, 3, xx, G.x().cc(), m->S + S_TMP, st);
    k_normalize<T><<<nb(n), EB, 0, st>>>(n, 3, P4<T>(G.x().cc(), 3), M4<T>(G.x().mm(), 3), m->S + S_TMP);
    ckl();
    for (int it = 0; it < m->opts.power_iters; ++it) {
      apply_K_level<T>(mesh, h, G.x().cc(), G.t.mm(), st);
      k_bmul<T><<<nb(n), EB, 0, st>>>(n, G.bi(), P4<T>(G.t.cc(), 3), M4<T>(G.d().mm(), 3));
      ckl();
      const T* const* dd[1] = {G.d().cc()};
      dots<T>(m, L, 1, 3, dd, G.d().cc(), m->S + S_TMP + h % 4, st);
      k_normalize<T><<<nb(n), EB, 0, st>>>(n, 3, P4<T>(G.d().cc(), 3), M4<T>(G.x().mm(), 3), m->S + S_TMP + h % 4);
      ckl();
    }
    double l2 = 0.0;
    ck(cudaMemcpyAsync(&l2, m->S + S_TMP + h % 4, sizeof(double), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    G.lam = std::sqrt(l2);
  }
  // Deflation of the constant pressure mode: under free-slip P B^T 1 != 0 at the boundary
  // nodes, so the constant pressure is a near-null (not null) mode of the Schur complement that
  // the diagonal Schur approximation misses.  S 1 = -B A^-1 c, c = P B^T 1, with A^-1 c from
  // two stationary V-cycle iterations.
  {
    const Level& L0 = mesh->lv[0];
    const Level& L1 = mesh->lv[1];
    MGLevelT<T>& G = P.L[0];
    const int64_t n0 = L0.n_layout, n1 = L1.n_layout;
    k_fill<T><<<nb(n1), EB, 0, st>>>(n1, (T)1, P.ones_p);
    ckl();
    T* scr = sizeof(T) == 8 ? (T*)L0.scr64 : (T*)L0.scr32;
    const T* cin[1] = {P.ones_p};
    T* fout[1] = {scr};
    ck(launch_prolong<T>(L0, L1, bc, 1, 0, cin, fout, st));
    ck(launch_grad_fine<T>(L0, bc, scr, G.r.mm(), st));  // c in G.r
    Vec3<T>& wv = P.defl_w;
    Vec3<T>& cc = P.defl_c;
    for (int q = 0; q < 3; ++q) ck(cudaMemcpyAsync(cc.c[q], G.r.c[q], sizeof(T) * n0, cudaMemcpyDeviceToDevice, st));
    for (int q = 0; q < 3; ++q) ck(cudaMemsetAsync(wv.c[q], 0, sizeof(T) * n0, st));
    for (int cyc = 0; cyc < 2; ++cyc) {
      // b = c - A w
      apply_K_level<T>(mesh, 0, wv.cc(), G.t.mm(), st);
      k_axpby<T><<<nb(n0), EB, 0, st>>>(n0, 3, 1.0, P4<T>(cc.cc(), 3), 0.0, M4<T>(G.b.mm(), 3));
      ckl();
      k_axpby<T><<<nb(n0), EB, 0, st>>>(n0, 3, -1.0, P4<T>(G.t.cc(), 3), 1.0, M4<T>(G.b.mm(), 3));
      ckl();
      vcycle_level<T>(m, mesh, 0, st);
      k_axpby<T><<<nb(n0), EB, 0, st>>>(n0, 3, 1.0, P4<T>(G.x().cc(), 3), 1.0, M4<T>(wv.mm(), 3));
      ckl();
    }
    ck(launch_div_fine<T>(L0, bc, wv.cc(), scr, st));
    const T* fin[1] = {scr};
    T* cout[1] = {P.sq};
    ck(launch_restrict<T>(L0, L1, bc, 1, 0, fin, cout, st));
    k_axpby<T><<<nb(n1), EB, 0, st>>>(n1, 1, 0.0, P4<T>((const T* const*)&P.sq, 1), -1.0, M4<T>(&P.sq, 1));
    ckl();
    const T* sqa[1] = {P.sq};
    const T* const* sqp[1] = {sqa};
    const T* on[1] = {P.ones_p};
    dots<T>(m, L1, 1, 1, sqp, on, m->S + S_TMP, st);
    const double qsq = host_scalar(m, S_TMP, st);
    // off when the constant pressure is (numerically) an exact null vector (no-slip on both surfaces)
    double cn = 0.0;
    const T* const* ccp[1] = {cc.cc()};
    dots<T>(m, L0, 1, 3, ccp, cc.cc(), m->S + S_TMP, st);
    cn = host_scalar(m, S_TMP, st);
    P.qsq = (cn > 0.0 && qsq != 0.0) ? qsq : 0.0;
  }
  ck(cudaStreamSynchronize(st));
  if (g_err != cudaSuccess) return TN_ECUDA;
  capture_vcycle<T>(m, mesh);
  if (g_err != cudaSuccess) return TN_ECUDA;
  P.ready = true;
  return TN_OK;
}

template <typename T>
void vcycle_t(tn_mesh* mesh, const T* const* r, T* const* z, cudaStream_t st) {
  MGState* m = mesh->mg;
  MGLevelT<T>& G = ps<T>(m).L[0];
  const int64_t n = mesh->lv[0].n_layout;
  for (int c = 0; c < 3; ++c) ck(cudaMemcpyAsync(G.b.c[c], r[c], sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
  run_vcycle<T>(m, mesh, st);
  for (int c = 0; c < 3; ++c) ck(cudaMemcpyAsync(z[c], G.x().c[c], sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
}

// ============================================================================ FGMRES
template <typename T>
void alloc_kvec(MGState* m, const tn_mesh* mesh, KVec<T>& v) {
  for (int c = 0; c < 3; ++c) v.u[c] = alloc_zero<T>(m, mesh->lv[0].n_layout);
  v.p = alloc_zero<T>(m, mesh->lv[1].n_layout);
}

template <typename T>
void ensure_krylov(MGState* m, const tn_mesh* mesh, int restart) {
  // restart 0: only V[0] and the work vectors (the FP64 side of the mixed mode)
  PrecState<T>& P = ps<T>(m);
  if ((int)P.Z.size() >= restart && !P.V.empty()) return;
  if ((int)P.V.size() < restart + 1) P.V.resize(restart + 1);
  if ((int)P.Z.size() < restart) P.Z.resize(restart);
  for (auto& v : P.V)
    if (!v.p) alloc_kvec<T>(m, mesh, v);
  for (auto& v : P.Z)
    if (!v.p) alloc_kvec<T>(m, mesh, v);
  if (!P.w.p) alloc_kvec<T>(m, mesh, P.w);
  if (!P.tmp.p) alloc_kvec<T>(m, mesh, P.tmp);
  if (sizeof(T) == 4 && !P.ir_r.p) alloc_kvec<T>(m, mesh, P.ir_r), alloc_kvec<T>(m, mesh, P.ir_c);
  if (!P.tu[0])
    for (int c = 0; c < 3; ++c) P.tu[c] = alloc_zero<T>(m, mesh->lv[0].n_layout);
}

// y = K x  (K = [[P A P + I - P, P B^T], [B P, 0]])
template <typename T>
void apply_K(MGState* m, tn_mesh* mesh, const KVec<T>& x, KVec<T>& y, cudaStream_t st) {
  PrecState<T>& P = ps<T>(m);
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  const BC bc{mesh->bc_in, mesh->bc_out};
  ck(launch_apply_A<T>(L0, bc, mesh->div_term, (const T* const*)x.u, (T* const*)y.u, st));
  T* scr = sizeof(T) == 8 ? (T*)L0.scr64 : (T*)L0.scr32;
  const T* cin[1] = {x.p};
  T* fout[1] = {scr};
  ck(launch_prolong<T>(L0, L1, bc, 1, 0, cin, fout, st));
  ck(launch_grad_fine<T>(L0, bc, scr, (T* const*)P.tu, st));
  k_axpby<T><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, 3, 1.0, P4<T>((const T* const*)P.tu, 3), 1.0,
                                             M4<T>((T* const*)y.u, 3));
  ckl();
  ck(launch_div_fine<T>(L0, bc, (const T* const*)x.u, scr, st));
  const T* fin[1] = {scr};
  T* cout[1] = {y.p};
  ck(launch_restrict<T>(L0, L1, bc, 1, 0, fin, cout, st));
}

// z = P^-1 r: z_p = -r_p / diag(M_1/eta), z_u = V(r_u - B^T z_p).  Split around the V-cycle for
// the lockstep solver: prec_pre (z_p and the V-cycle's right-hand side), the V-cycle, prec_post.
template <typename T>
void prec_pre(MGState* m, tn_mesh* mesh, const KVec<T>& r, KVec<T>& z, cudaStream_t st) {
  PrecState<T>& P = ps<T>(m);
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  const BC bc{mesh->bc_in, mesh->bc_out};
  if (P.qsq != 0.0) {
    const T* rr[1] = {r.p};
    const T* const* rp[1] = {rr};
    const T* on[1] = {P.ones_p};
    dots<T>(m, L1, 1, 1, rp, on, m->S + S_QR, st);
    k_schur_defl<T><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, P.mdiag, r.p, P.sq, m->S + S_QR, 1.0 / P.qsq, z.p);
  } else {
    k_schur<T><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, P.mdiag, r.p, z.p);
  }
  ckl();
  T* scr = sizeof(T) == 8 ? (T*)L0.scr64 : (T*)L0.scr32;
  const T* cin[1] = {z.p};
  T* fout[1] = {scr};
  ck(launch_prolong<T>(L0, L1, bc, 1, 0, cin, fout, st));
  ck(launch_grad_fine<T>(L0, bc, scr, (T* const*)P.tu, st));
  MGLevelT<T>& G = P.L[0];
  k_axpby<T><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, 3, 1.0, P4<T>((const T* const*)r.u, 3), 0.0,
                                             M4<T>(G.b.mm(), 3));
  ckl();
  k_axpby<T><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, 3, -1.0, P4<T>((const T* const*)P.tu, 3), 1.0,
                                             M4<T>(G.b.mm(), 3));
  ckl();
}

template <typename T>
void prec_post(MGState* m, tn_mesh* mesh, KVec<T>& z, cudaStream_t st) {
  PrecState<T>& P = ps<T>(m);
  const Level& L0 = mesh->lv[0];
  MGLevelT<T>& G = P.L[0];
  for (int c = 0; c < 3; ++c)
    ck(cudaMemcpyAsync(z.u[c], G.x().c[c], sizeof(T) * L0.n_layout, cudaMemcpyDeviceToDevice, st));
}

template <typename T>
void apply_prec(MGState* m, tn_mesh* mesh, const KVec<T>& r, KVec<T>& z, cudaStream_t st) {
  prec_pre<T>(m, mesh, r, z, st);
  run_vcycle<T>(m, mesh, st);
  prec_post<T>(m, mesh, z, st);
}


// FP64 Krylov vector -> FP32 preconditioner -> FP64 (mode TN_SOLVE_F64_PREC32): the vector is
// unit-norm, so FP32 holds it without scaling.
void prec_f32_pre(MGState* m, tn_mesh* mesh, const KVec<double>& r, cudaStream_t st) {
  PrecState<float>& F = m->p32;
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  for (int c = 0; c < 3; ++c) {
    k_convert<double, float><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, r.u[c], F.ir_r.u[c], 1.0);
    ckl();
  }
  k_convert<double, float><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, r.p, F.ir_r.p, 1.0);
  ckl();
  prec_pre<float>(m, mesh, F.ir_r, F.ir_c, st);
}

void prec_f32_post(MGState* m, tn_mesh* mesh, KVec<double>& z, cudaStream_t st) {
  PrecState<float>& F = m->p32;
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  prec_post<float>(m, mesh, F.ir_c, st);
  for (int c = 0; c < 3; ++c) {
    k_convert<float, double><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, F.ir_c.u[c], z.u[c], 1.0);
    ckl();
  }
  k_convert<float, double><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, F.ir_c.p, z.p, 1.0);
  ckl();
}

void apply_prec_f32(MGState* m, tn_mesh* mesh, const KVec<double>& r, KVec<double>& z, cudaStream_t st) {
  prec_f32_pre(m, mesh, r, st);
  run_vcycle<float>(m, mesh, st);
  prec_f32_post(m, mesh, z, st);
}

// Restarted FGMRES(m) with right preconditioning and CGS2 orthogonalisation (Saad 1993).
// Solves K x = b from the given x; stops when ||b - K x|| <= abstol (recurrence estimate,
// confirmed by the true residual at every restart) or after max_iters.  Returns the
// iterations used; *res gets the final true residual norm.
// Breakdown exits (*brk): FGMRES_NONFINITE at once when the restart residual or a Hessenberg
// column is not finite (x keeps only the finite columns' update); FGMRES_STALL after
// kStallRestarts restarts in a row that bring the residual less than 0.1 % below its best so far;
// FGMRES_CANCELLED when the mesh's cancel flag is set (checked once per iteration).
enum { FGMRES_OK = 0, FGMRES_NONFINITE = 1, FGMRES_STALL = 2, FGMRES_CANCELLED = 3 };
constexpr int kStallRestarts = 5;

bool cancelled(const tn_mesh* mesh) {
  return mesh->cancel && mesh->cancel->load(std::memory_order_relaxed) != 0;
}

template <typename T>
int fgmres(MGState* m, tn_mesh* mesh, const KVec<T>& b, KVec<T>& x, double abstol, int restart, int max_iters,
           double* res, cudaStream_t st, bool prec32 = false, int* brk = nullptr) {
  PrecState<T>& P = ps<T>(m);
  ensure_krylov<T>(m, mesh, restart);
  int its = 0, stall = 0, why = FGMRES_OK;
  std::vector<double> H((restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart);
  double beta = 0, beta_best = 0;
  while (true) {
    // r = b - K x  -> V[0]
    apply_K<T>(m, mesh, x, P.w, st);
    kaxpby<T>(mesh, 1.0, b, 0.0, P.V[0], st);
    kaxpby<T>(mesh, -1.0, P.w, 1.0, P.V[0], st);
    const KVec<T>* v0[1] = {&P.V[0]};
    kdots<T>(m, mesh, 1, v0, P.V[0], m->S + S_NRM, st);
    beta = std::sqrt(host_scalar(m, S_NRM, st));
    *res = beta;
    // progress is measured against the best restart residual so far: at the rounding floor the
    // residual fluctuates, and a comparison with the previous restart alone would keep resetting
    if (!std::isfinite(beta)) why = FGMRES_NONFINITE;
    else if (its > 0 && !(beta < 0.999 * beta_best)) ++stall;
    else stall = 0;
    if (stall >= kStallRestarts) why = FGMRES_STALL;
    if (cancelled(mesh)) why = FGMRES_CANCELLED;
    if (its == 0 || beta < beta_best) beta_best = beta;
    if (why != FGMRES_OK || beta <= abstol || its >= max_iters || g_err != cudaSuccess) break;
    kaxpby<T>(mesh, 0.0, P.V[0], 1.0 / beta, P.V[0], st);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < restart && its < max_iters; ++j) {
      if constexpr (sizeof(T) == 8) {
        if (prec32) apply_prec_f32(m, mesh, P.V[j], P.Z[j], st);
        else apply_prec<T>(m, mesh, P.V[j], P.Z[j], st);
      } else {
        apply_prec<T>(m, mesh, P.V[j], P.Z[j], st);
      }
      apply_K<T>(m, mesh, P.Z[j], P.w, st);
      std::vector<const KVec<T>*> vb(j + 1);
      for (int i = 0; i <= j; ++i) vb[i] = &P.V[i];
      kdots<T>(m, mesh, j + 1, vb.data(), P.w, m->S + S_H, st);
      kaxpy<T>(mesh, j + 1, vb.data(), m->S + S_H, -1.0, P.w, st);
      kdots<T>(m, mesh, j + 1, vb.data(), P.w, m->S + S_H2, st);
      kaxpy<T>(mesh, j + 1, vb.data(), m->S + S_H2, -1.0, P.w, st);
      const KVec<T>* wv[1] = {&P.w};
      kdots<T>(m, mesh, 1, wv, P.w, m->S + S_NRM, st);
      double hs[S_MAX];
      ck(cudaMemcpyAsync(hs, m->S, sizeof(double) * S_MAX, cudaMemcpyDeviceToHost, st));
      ck(cudaStreamSynchronize(st));
      double* col = &H[j * (restart + 1)];
      bool finite = std::isfinite(hs[S_NRM]);
      for (int i = 0; i <= j; ++i) {
        col[i] = hs[S_H + i] + hs[S_H2 + i];
        finite = finite && std::isfinite(col[i]);
      }
      if (!finite) {  // this column is unusable: update x with the previous ones and stop
        why = FGMRES_NONFINITE;
        break;
      }
      const double hn = std::sqrt(hs[S_NRM]);
      col[j + 1] = hn;
      if (hn > 0) kaxpby<T>(mesh, 1.0 / hn, P.w, 0.0, P.V[j + 1], st);
      for (int i = 0; i < j; ++i) {  // previous Givens rotations
        const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t0;
      }
      const double den = std::sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
      cs[j] = den > 0 ? col[j] / den : 1.0;
      sn[j] = den > 0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      if (std::fabs(g[j + 1]) <= abstol || hn == 0.0 || g_err != cudaSuccess || cancelled(mesh)) {
        ++j;
        break;
      }
    }
    // y = H^-1 g, x += Z y
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[k * (restart + 1) + i] * y[k];
      y[i] = s / H[i * (restart + 1) + i];
    }
    ck(cudaMemcpyAsync(m->S + S_Y, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
    std::vector<const KVec<T>*> zb(j);
    for (int i = 0; i < j; ++i) zb[i] = &P.Z[i];
    if (j > 0) kaxpy<T>(mesh, j, zb.data(), m->S + S_Y, 1.0, x, st);
    ck(cudaStreamSynchronize(st));
    if (why != FGMRES_OK) break;
  }
  if (brk) *brk = why;
  return its;
}

const char* breakdown_text(int why) {
  switch (why) {
    case FGMRES_NONFINITE: return "breakdown: non-finite residual or Hessenberg entry (NaN / Inf in the operator or data)";
    case FGMRES_STALL: return "stagnation: five restarts in a row without a new residual minimum (0.1 % below the best)";
    case FGMRES_CANCELLED: return "cancelled";
    default: return "not converged";
  }
}

// ---------------------------------------------------------------- lockstep FGMRES (serving batches)
// Several systems advance in lockstep on one stream: each round enqueues, for every system, either
// its restart residual or one FGMRES iteration, launches the V-cycles of all iterating systems
// together as one CUDA graph (each system's captured V-cycle a child graph, run concurrently),
// synchronises once and does every system's host part.  Per system the enqueued kernels, their
// order and the host arithmetic are those of fgmres<double>, so each result is bitwise the one of
// a solve alone.
struct LockSys {
  tn_mesh* mesh = nullptr;
  MGState* m = nullptr;
  KVec<double> b, x;
  double abstol = 0, beta = 0, beta_best = 0;
  int its = 0, j = 0, stall = 0, why = FGMRES_OK, phase = 0;  // phase 0 restart, 1 iterating, 2 done
  std::vector<double> H, cs, sn, g, y;
  double* hs = nullptr;  // pinned host copy of the system's device scalars
};

cudaGraph_t sys_vtemplate(MGState* m, bool prec32) { return prec32 ? m->p32.vtemplate : m->p64.vtemplate; }

// The combined V-cycle graph of a subset of systems (bit mask), instantiated once and cached.
struct VcycleBatch {
  std::vector<std::pair<uint64_t, cudaGraphExec_t>> cache;
  ~VcycleBatch() {
    for (auto& c : cache) cudaGraphExecDestroy(c.second);
  }
  cudaGraphExec_t get(uint64_t mask, std::vector<LockSys>& sys, bool prec32) {
    for (auto& c : cache)
      if (c.first == mask) return c.second;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return nullptr;
    bool ok = true;
    for (size_t i = 0; i < sys.size() && ok; ++i) {
      if (!(mask >> i & 1)) continue;
      cudaGraph_t child = sys_vtemplate(sys[i].m, prec32);
      cudaGraphNode_t node;
      ok = child && cudaGraphAddChildGraphNode(&node, g, nullptr, 0, child) == cudaSuccess;
    }
    if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (ex) cache.emplace_back(mask, ex);
    return ex;
  }
};

void lock_update_x(LockSys& q, int cols, int rs, cudaStream_t st) {
  PrecState<double>& P = q.m->p64;
  for (int i = cols - 1; i >= 0; --i) {
    double v = q.g[i];
    for (int k = i + 1; k < cols; ++k) v -= q.H[k * (rs + 1) + i] * q.y[k];
    q.y[i] = v / q.H[i * (rs + 1) + i];
  }
  ck(cudaMemcpyAsync(q.m->S + S_Y, q.y.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st));
  std::vector<const KVec<double>*> zb(cols);
  for (int i = 0; i < cols; ++i) zb[i] = &P.Z[i];
  if (cols > 0) kaxpy<double>(q.mesh, cols, zb.data(), q.m->S + S_Y, 1.0, q.x, st);
}

void fgmres_lockstep(std::vector<LockSys>& sys, int restart, int max_iters, bool prec32, cudaStream_t st) {
  VcycleBatch vb;
  for (auto& q : sys) {
    q.H.assign((restart + 1) * restart, 0.0);
    q.cs.assign(restart, 0.0), q.sn.assign(restart, 0.0), q.g.assign(restart + 1, 0.0), q.y.assign(restart, 0.0);
  }
  while (g_err == cudaSuccess) {
    bool any = false;
    uint64_t mask = 0;
    // enqueue: restart residuals, and the first half of an iteration up to the V-cycle
    for (size_t i = 0; i < sys.size(); ++i) {
      LockSys& q = sys[i];
      PrecState<double>& P = q.m->p64;
      if (q.phase == 2) continue;
      any = true;
      if (q.phase == 0) {
        apply_K<double>(q.m, q.mesh, q.x, P.w, st);
        kaxpby<double>(q.mesh, 1.0, q.b, 0.0, P.V[0], st);
        kaxpby<double>(q.mesh, -1.0, P.w, 1.0, P.V[0], st);
        const KVec<double>* v0[1] = {&P.V[0]};
        kdots<double>(q.m, q.mesh, 1, v0, P.V[0], q.m->S + S_NRM, st);
        ck(cudaMemcpyAsync(q.hs, q.m->S, sizeof(double) * S_MAX, cudaMemcpyDeviceToHost, st));
      } else {
        if (prec32) prec_f32_pre(q.m, q.mesh, P.V[q.j], st);
        else prec_pre<double>(q.m, q.mesh, P.V[q.j], P.Z[q.j], st);
        mask |= (uint64_t)1 << i;
      }
    }
    if (!any) break;
    if (mask) {
      cudaGraphExec_t ex = (mask & (mask - 1)) ? vb.get(mask, sys, prec32) : nullptr;
      if (ex) {
        ck(cudaGraphLaunch(ex, st));
      } else {
        for (size_t i = 0; i < sys.size(); ++i)
          if (mask >> i & 1) {
            if (prec32) run_vcycle<float>(sys[i].m, sys[i].mesh, st);
            else run_vcycle<double>(sys[i].m, sys[i].mesh, st);
          }
      }
    }
    // second half of the iterations: preconditioned vector, operator, CGS2
    for (size_t i = 0; i < sys.size(); ++i) {
      if (!(mask >> i & 1)) continue;
      LockSys& q = sys[i];
      PrecState<double>& P = q.m->p64;
      const int j = q.j;
      if (prec32) prec_f32_post(q.m, q.mesh, P.Z[j], st);
      else prec_post<double>(q.m, q.mesh, P.Z[j], st);
      apply_K<double>(q.m, q.mesh, P.Z[j], P.w, st);
      std::vector<const KVec<double>*> vbs(j + 1);
      for (int k = 0; k <= j; ++k) vbs[k] = &P.V[k];
      kdots<double>(q.m, q.mesh, j + 1, vbs.data(), P.w, q.m->S + S_H, st);
      kaxpy<double>(q.mesh, j + 1, vbs.data(), q.m->S + S_H, -1.0, P.w, st);
      kdots<double>(q.m, q.mesh, j + 1, vbs.data(), P.w, q.m->S + S_H2, st);
      kaxpy<double>(q.mesh, j + 1, vbs.data(), q.m->S + S_H2, -1.0, P.w, st);
      const KVec<double>* wv[1] = {&P.w};
      kdots<double>(q.m, q.mesh, 1, wv, P.w, q.m->S + S_NRM, st);
      ck(cudaMemcpyAsync(q.hs, q.m->S, sizeof(double) * S_MAX, cudaMemcpyDeviceToHost, st));
    }
    ck(cudaStreamSynchronize(st));
    if (g_err != cudaSuccess) break;
    // host part of every system, in order
    for (size_t i = 0; i < sys.size(); ++i) {
      LockSys& q = sys[i];
      PrecState<double>& P = q.m->p64;
      if (q.phase == 0) {
        q.beta = std::sqrt(q.hs[S_NRM]);
        if (!std::isfinite(q.beta)) q.why = FGMRES_NONFINITE;
        else if (q.its > 0 && !(q.beta < 0.999 * q.beta_best)) ++q.stall;
        else q.stall = 0;
        if (q.stall >= kStallRestarts) q.why = FGMRES_STALL;
        if (cancelled(q.mesh)) q.why = FGMRES_CANCELLED;
        if (q.its == 0 || q.beta < q.beta_best) q.beta_best = q.beta;
        if (q.why != FGMRES_OK || q.beta <= q.abstol || q.its >= max_iters) {
          q.phase = 2;
          continue;
        }
        kaxpby<double>(q.mesh, 0.0, P.V[0], 1.0 / q.beta, P.V[0], st);
        std::fill(q.g.begin(), q.g.end(), 0.0);
        q.g[0] = q.beta;
        q.j = 0;
        q.phase = 1;
        continue;
      }
      if (q.phase != 1) continue;
      const int j = q.j;
      double* col = &q.H[j * (restart + 1)];
      bool finite = std::isfinite(q.hs[S_NRM]);
      for (int k = 0; k <= j; ++k) {
        col[k] = q.hs[S_H + k] + q.hs[S_H2 + k];
        finite = finite && std::isfinite(col[k]);
      }
      if (!finite) {  // update x with the previous columns and stop
        q.why = FGMRES_NONFINITE;
        lock_update_x(q, j, restart, st);
        q.phase = 2;
        continue;
      }
      const double hn = std::sqrt(q.hs[S_NRM]);
      col[j + 1] = hn;
      if (hn > 0) kaxpby<double>(q.mesh, 1.0 / hn, P.w, 0.0, P.V[j + 1], st);
      for (int k = 0; k < j; ++k) {
        const double t0 = q.cs[k] * col[k] + q.sn[k] * col[k + 1];
        col[k + 1] = -q.sn[k] * col[k] + q.cs[k] * col[k + 1];
        col[k] = t0;
      }
      const double den = std::sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
      q.cs[j] = den > 0 ? col[j] / den : 1.0;
      q.sn[j] = den > 0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      q.g[j + 1] = -q.sn[j] * q.g[j];
      q.g[j] = q.cs[j] * q.g[j];
      ++q.its;
      const bool stop = std::fabs(q.g[j + 1]) <= q.abstol || hn == 0.0 || cancelled(q.mesh);
      if (stop || j + 1 >= restart || q.its >= max_iters) {  // end of the cycle: x += Z y, then restart
        lock_update_x(q, j + 1, restart, st);
        q.phase = 0;
      } else {
        q.j = j + 1;
      }
    }
  }
}

template <typename T>
KVec<T> wrap(T* const* u, T* p) {
  KVec<T> v;
  for (int c = 0; c < 3; ++c) v.u[c] = u[c];
  v.p = p;
  return v;
}

}  // namespace

// Multigrid level shapes (lateral level, node layers) from the mesh's level 0 down.  A cell's
// radial / lateral size ratio q = (r_out - r_in) 2^l / (atan(2) r_mid (N_r - 1)) (atan(2): the
// angle between neighbouring icosahedron vertices, r_mid the mid radius) decides the next
// level: q >= 2 coarsens laterally only, q <= 1/2 radially only, otherwise both directions
// (or the one still possible); the hierarchy ends when the preferred direction cannot coarsen.
std::vector<std::pair<int, int>> mg_shapes(int l0, int nr0, double r_in, double r_out) {
  std::vector<std::pair<int, int>> out{{l0, nr0}};
  const double edge = 1.1071487177940904;
  while (true) {
    const int l = out.back().first, nr = out.back().second, R = nr - 1;
    const bool can_lat = l >= 2, can_rad = R % 2 == 0 && R >= 2;
    const double q = (r_out - r_in) * (double)(1 << l) / (edge * (0.5 * (r_in + r_out)) * (double)R);
    int nl = l, nn = nr;
    if (q >= 2.0) {
      if (!can_lat) break;
      nl = l - 1;
    } else if (q <= 0.5) {
      if (!can_rad) break;
      nn = R / 2 + 1;
    } else if (can_lat && can_rad) {
      nl = l - 1, nn = R / 2 + 1;
    } else if (can_lat) {
      nl = l - 1;
    } else if (can_rad) {
      nn = R / 2 + 1;
    } else {
      break;
    }
    out.push_back({nl, nn});
  }
  return out;
}

void mg_free(MGState* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  for (Level* L : m->owned_levels) {
    destroy_level(*L);
    delete L;
  }
  if (m->p64.vgraph) cudaGraphExecDestroy(m->p64.vgraph);
  if (m->p32.vgraph) cudaGraphExecDestroy(m->p32.vgraph);
  if (m->p64.vtemplate) cudaGraphDestroy(m->p64.vtemplate);
  if (m->p32.vtemplate) cudaGraphDestroy(m->p32.vtemplate);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->S) cudaFree(m->S);
  if (m->flag) cudaFree(m->flag);
  if (m->part) cudaFree(m->part);
  delete m;
}

void mg_invalidate(tn_mesh* mesh) {
  if (mesh->mg) mesh->mg->p64.ready = mesh->mg->p32.ready = false;
}

}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_mg_default_opts(tn_mg_opts* o) {
  if (!o) return TN_EINVAL;
  o->pre_smooth = 2;
  o->post_smooth = 2;
  o->cheb_degree = 2;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->power_iters = 15;
  o->coarse_max_iters = 50;
  o->coarse_rtol = 1e-3;
  o->levels = 0;
  o->seed = 0x5eedull;
  return TN_OK;
}

tn_status tn_mg_setup(tn_mesh* mesh, tn_prec prec, const tn_mg_opts* opts, const void* const* v0, void* stream) {
  if (!mesh) return TN_EINVAL;
  if (!mesh->eta_set) {
    set_error("tn_mg_setup: viscosity not set");
    return TN_ESTATE;
  }
  if (mesh->lv.size() < 2) {
    set_error("tn_mg_setup: the mesh hierarchy has a single level");
    return TN_EINVAL;
  }
  tn_mg_opts o;
  tn_mg_default_opts(&o);
  if (opts) o = *opts;
  if (o.cheb_degree != 2 || o.pre_smooth < 0 || o.post_smooth < 0 || o.power_iters < 1 || o.coarse_max_iters < 1 ||
      !(o.cheb_hi > o.cheb_lo) || !(o.cheb_lo > 0)) {
    set_error("tn_mg_setup: invalid multigrid options");
    return TN_EINVAL;
  }
  const std::vector<std::pair<int, int>> shapes = mg_shapes(mesh->lv[0].l, mesh->lv[0].n_r, mesh->r_in, mesh->r_out);
  const int avail = (int)shapes.size();
  const int nlev = o.levels <= 0 ? avail : std::min(o.levels, avail);
  if (nlev < 2) {
    set_error("tn_mg_setup: need at least two levels");
    return TN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  g_err = cudaSuccess;
  MGState* m = mesh->mg;
  if (m && (m->nlev != nlev)) {
    mg_free(m);
    mesh->mg = m = nullptr;
  }
  if (!m) {
    m = new MGState();
    m->nlev = nlev;
    // level geometry: the mesh's levels while the multigrid coarsens fully, own levels after
    bool same = true;
    for (int h = 0; h < nlev; ++h) {
      same = same && h < (int)mesh->lv.size() && mesh->lv[h].l == shapes[h].first &&
             mesh->lv[h].n_r == shapes[h].second;
      if (same) {
        m->geo.push_back(&mesh->lv[h]);
        continue;
      }
      Level* L = new Level();
      tn_status cs = create_level(*L, shapes[h].first, shapes[h].second, mesh->r_in, mesh->r_out, mesh->eta_storage,
                                  mesh->div_term);
      L->hg_kappa = mesh->hg_kappa;
      L->quad = mesh->quad;
      L->df = mesh->df;
      m->owned_levels.push_back(L);
      if (cs != TN_OK) {
        mesh->mg = m;
        mg_free(m);
        mesh->mg = nullptr;
        return cs;
      }
      m->geo.push_back(L);
    }
    ck(cudaMalloc((void**)&m->S, sizeof(double) * S_MAX));
    ck(cudaMemset(m->S, 0, sizeof(double) * S_MAX));
    ck(cudaMalloc((void**)&m->flag, sizeof(int)));
    ck(cudaMalloc((void**)&m->part, sizeof(double) * 2 * MAXV * RG));
    mesh->mg = m;
    if (g_err != cudaSuccess) {
      set_error("tn_mg_setup: device allocation failed");
      return TN_ENOMEM;
    }
  }
  m->opts = o;
  // viscosity of the multigrid's own levels: mean of the children on the level above
  for (int h = 1; h < m->nlev; ++h) {
    if (m->geo[h] == &mesh->lv[h]) continue;
    ck(launch_eta_coarsen(*m->geo[h - 1], *m->geo[h], m->geo[h - 1]->eta64, m->geo[h]->eta64, st));
    ck(launch_eta_f32_path(*m->geo[h], st));
  }
  tn_status s = prec == TN_F64 ? mg_setup_t<double>(mesh, v0, st) : mg_setup_t<float>(mesh, v0, st);
  if (s != TN_OK) set_error(std::string("tn_mg_setup: ") + cudaGetErrorString(g_err));
  return s;
}

tn_status tn_mg_lambda(const tn_mesh* mesh, tn_prec prec, int level, double* lam) {
  if (!mesh || !mesh->mg || !lam || level < 0 || level >= mesh->mg->nlev) return TN_EINVAL;
  if (prec == TN_F64) {
    if (mesh->mg->p64.L.empty()) return TN_ESTATE;
    *lam = mesh->mg->p64.L[level].lam;
  } else {
    if (mesh->mg->p32.L.empty()) return TN_ESTATE;
    *lam = mesh->mg->p32.L[level].lam;
  }
  return TN_OK;
}

tn_status tn_vcycle(tn_mesh* mesh, tn_prec prec, const void* const* r, void* const* z, void* stream) {
  if (!mesh || !r || !z) return TN_EINVAL;
  for (int c = 0; c < 3; ++c)
    if (!r[c] || !z[c] || r[c] == z[c]) {
      set_error("tn_vcycle: NULL or aliased vectors");
      return TN_EINVAL;
    }
  if (!mesh->mg || !(prec == TN_F64 ? mesh->mg->p64.ready : mesh->mg->p32.ready)) {
    tn_status s = tn_mg_setup(mesh, prec, mesh->mg ? &mesh->mg->opts : nullptr, nullptr, stream);
    if (s != TN_OK) return s;
  }
  g_err = cudaSuccess;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == TN_F64) vcycle_t<double>(mesh, (const double* const*)r, (double* const*)z, st);
  else vcycle_t<float>(mesh, (const float* const*)r, (float* const*)z, st);
  if (g_err != cudaSuccess) {
    set_error(std::string("tn_vcycle: ") + cudaGetErrorString(g_err));
    return TN_ECUDA;
  }
  return TN_OK;
}

tn_status tn_solve_default_opts(tn_solve_opts* o) {
  if (!o) return TN_EINVAL;
  o->rtol = 1e-8;
  o->restart = 30;
  o->max_iters = 2000;
  o->mode = TN_SOLVE_F64;
  o->inner_rtol = 1e-3;
  o->inner_max_iters = 100;
  o->max_refinements = 30;
  return TN_OK;
}

}  // extern "C"

namespace {

// Checks shared by the single and the batched solve.
tn_status solve_check(const char* who, tn_mesh* mesh, const tn_solve_opts& o, const double* const* f,
                      double* const* u, double* p) {
  if (!mesh || !f || !u || !p) {
    set_error(std::string(who) + ": NULL argument");
    return TN_EINVAL;
  }
  for (int c = 0; c < 3; ++c)
    if (!f[c] || !u[c]) {
      set_error(std::string(who) + ": NULL vector");
      return TN_EINVAL;
    }
  if (mesh->lv.size() < 2) {
    set_error(std::string(who) + ": the mesh hierarchy has a single level");
    return TN_EINVAL;
  }
  if (o.restart < 1 || o.restart > MAX_RESTART || !(o.rtol > 0) || o.max_iters < 1 ||
      (o.mode != TN_SOLVE_F64 && o.mode != TN_SOLVE_MIXED && o.mode != TN_SOLVE_F64_PREC32)) {
    set_error(std::string(who) + ": invalid options (restart must be in [1, 30])");
    return TN_EINVAL;
  }
  return TN_OK;
}

// Multigrid set-up when needed, workspaces, b = (f, g) in the FP64 temporary, x = (u, p) = 0 and
// ||b|| (one host synchronisation).
tn_status solve_begin(tn_mesh* mesh, const tn_solve_opts& o, const double* const* f, const double* g, double* const* u,
                      double* p, cudaStream_t st, void* stream, KVec<double>& b, KVec<double>& x, double& bnorm) {
  const bool mixed = o.mode == TN_SOLVE_MIXED, prec32 = o.mode == TN_SOLVE_F64_PREC32;
  // the mixed modes need only the FP32 multigrid; the refinement mode keeps only the residual
  // work vectors in FP64, the FP32-preconditioner mode the FP64 Krylov basis
  const bool mg32 = mixed || prec32;
  if (!mesh->mg || !(mg32 ? mesh->mg->p32.ready : mesh->mg->p64.ready)) {
    const tn_status s = tn_mg_setup(mesh, mg32 ? TN_F32 : TN_F64, mesh->mg ? &mesh->mg->opts : nullptr, nullptr, stream);
    if (s != TN_OK) return s;
  }
  MGState* m = mesh->mg;
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  ensure_krylov<double>(m, mesh, mixed ? 0 : o.restart);
  if (mixed) ensure_krylov<float>(m, mesh, o.restart);
  if (prec32) ensure_krylov<float>(m, mesh, 0);
  if (g_err != cudaSuccess) {
    set_error("tn_stokes_solve: workspace allocation failed");
    return TN_ENOMEM;
  }
  b = m->p64.tmp;
  for (int c = 0; c < 3; ++c) ck(cudaMemcpyAsync(b.u[c], f[c], sizeof(double) * L0.n_layout, cudaMemcpyDeviceToDevice, st));
  if (g) ck(cudaMemcpyAsync(b.p, g, sizeof(double) * L1.n_layout, cudaMemcpyDeviceToDevice, st));
  else ck(cudaMemsetAsync(b.p, 0, sizeof(double) * L1.n_layout, st));
  x = wrap<double>(u, p);
  for (int c = 0; c < 3; ++c) ck(cudaMemsetAsync(u[c], 0, sizeof(double) * L0.n_layout, st));
  ck(cudaMemsetAsync(p, 0, sizeof(double) * L1.n_layout, st));
  const KVec<double>* bb[1] = {&b};
  kdots<double>(m, mesh, 1, bb, b, m->S + S_NRM, st);
  bnorm = std::sqrt(host_scalar(m, S_NRM, st));
  return TN_OK;
}

// Rigid rotations out of the returned velocity (free-slip on both surfaces), the true residual
// ||b - K x|| (one host synchronisation).
double solve_true_residual(tn_mesh* mesh, const KVec<double>& b, KVec<double>& x, cudaStream_t st) {
  MGState* m = mesh->mg;
  PrecState<double>& D = m->p64;
  if (rotations_singular(mesh)) project_rotations<double>(m, mesh->lv[0], x.u, st);
  KVec<double>& r = D.V[0];
  apply_K<double>(m, mesh, x, D.w, st);
  kaxpby<double>(mesh, 1.0, b, 0.0, r, st);
  kaxpby<double>(mesh, -1.0, D.w, 1.0, r, st);
  const KVec<double>* rv[1] = {&r};
  kdots<double>(m, mesh, 1, rv, r, m->S + S_NRM, st);
  return std::sqrt(host_scalar(m, S_NRM, st));
}

tn_status solve_status(const char* who, const tn_solve_opts& o, int its, int refs, int why, double res, double bnorm,
                       double seconds, tn_solve_stats* stats) {
  const double rel = bnorm > 0 ? res / bnorm : 0.0;
  if (stats) {
    stats->iterations = its;
    stats->refinements = refs;
    stats->rel_residual = rel;
    stats->seconds = seconds;
    stats->converged = why == FGMRES_OK && rel <= o.rtol;
  }
  if (g_err != cudaSuccess) {
    set_error(std::string(who) + ": " + cudaGetErrorString(g_err));
    return TN_ECUDA;
  }
  if (why == FGMRES_CANCELLED) {
    set_error(std::string(who) + ": cancelled");
    return TN_ECANCELED;
  }
  if (why != FGMRES_OK || !(rel <= o.rtol)) {  // !(<=): a NaN residual is not convergence
    set_error(std::string(who) + ": " + breakdown_text(why));
    return TN_ENOTCONVERGED;
  }
  return TN_OK;
}

}  // namespace

extern "C" {

tn_status tn_stokes_solve(tn_mesh* mesh, const tn_solve_opts* opts, const double* const* f, const double* g,
                          double* const* u, double* p, tn_solve_stats* stats, void* stream) {
  tn_solve_opts o;
  tn_solve_default_opts(&o);
  if (opts) o = *opts;
  tn_status s = solve_check("tn_stokes_solve", mesh, o, f, u, p);
  if (s != TN_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  const bool mixed = o.mode == TN_SOLVE_MIXED;
  const bool prec32 = o.mode == TN_SOLVE_F64_PREC32;
  g_err = cudaSuccess;
  KVec<double> b, x;
  double bnorm = 0;
  s = solve_begin(mesh, o, f, g, u, p, st, stream, b, x, bnorm);
  if (s != TN_OK) return s;
  MGState* m = mesh->mg;
  const Level& L0 = mesh->lv[0];
  const Level& L1 = mesh->lv[1];
  PrecState<double>& D = m->p64;
  int its = 0, refs = 0, why = FGMRES_OK;
  double res = bnorm;
  if (!std::isfinite(bnorm)) why = FGMRES_NONFINITE;  // NaN / Inf in f or g: nothing to solve
  if (bnorm > 0 && why == FGMRES_OK) {
    if (!mixed) {
      its = fgmres<double>(m, mesh, b, x, o.rtol * bnorm, o.restart, o.max_iters, &res, st, prec32, &why);
    } else {
      // FP64 iterative refinement around FP32 FGMRES / V-cycle inner solves
      PrecState<float>& F = m->p32;
      KVec<double>& r = D.V[0];
      KVec<float>& rr32 = F.ir_r;
      KVec<float>& c32 = F.ir_c;
      while (refs < o.max_refinements && its < o.max_iters) {
        apply_K<double>(m, mesh, x, D.w, st);
        kaxpby<double>(mesh, 1.0, b, 0.0, r, st);
        kaxpby<double>(mesh, -1.0, D.w, 1.0, r, st);
        const KVec<double>* rv[1] = {&r};
        kdots<double>(m, mesh, 1, rv, r, m->S + S_NRM, st);
        res = std::sqrt(host_scalar(m, S_NRM, st));
        if (!std::isfinite(res)) why = FGMRES_NONFINITE;
        else if (cancelled(mesh)) why = FGMRES_CANCELLED;
        if (why != FGMRES_OK || res <= o.rtol * bnorm || g_err != cudaSuccess) break;
        for (int c = 0; c < 3; ++c) {
          k_convert<double, float><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, r.u[c], rr32.u[c], 1.0 / res);
          ckl();
          ck(cudaMemsetAsync(c32.u[c], 0, sizeof(float) * L0.n_layout, st));
        }
        k_convert<double, float><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, r.p, rr32.p, 1.0 / res);
        ckl();
        ck(cudaMemsetAsync(c32.p, 0, sizeof(float) * L1.n_layout, st));
        double ires = 0;
        int iwhy = FGMRES_OK;
        its += fgmres<float>(m, mesh, rr32, c32, o.inner_rtol, o.restart, o.inner_max_iters, &ires, st, false, &iwhy);
        // an inner stall only ends this refinement step; non-finite values or a cancel end the solve
        if (iwhy == FGMRES_NONFINITE || iwhy == FGMRES_CANCELLED) {
          why = iwhy;
          break;
        }
        for (int c = 0; c < 3; ++c) {
          k_accum<float><<<nb(L0.n_layout), EB, 0, st>>>(L0.n_layout, c32.u[c], x.u[c], res);
          ckl();
        }
        k_accum<float><<<nb(L1.n_layout), EB, 0, st>>>(L1.n_layout, c32.p, x.p, res);
        ckl();
        ++refs;
      }
    }
    res = solve_true_residual(mesh, b, x, st);
  }
  ck(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return solve_status("tn_stokes_solve", o, its, refs, why, res, bnorm, secs, stats);
}

tn_status tn_stokes_solve_batch(tn_mesh* const* meshes, int n, const tn_solve_opts* opts, const double* const* const* f,
                                const double* const* g, double* const* const* u, double* const* p,
                                tn_solve_stats* stats, tn_status* status, void* stream) {
  if (!meshes || n < 1 || n > 64 || !f || !u || !p || !status) {
    set_error("tn_stokes_solve_batch: bad arguments (1 <= n <= 64)");
    return TN_EINVAL;
  }
  tn_solve_opts o;
  tn_solve_default_opts(&o);
  if (opts) o = *opts;
  if (o.mode == TN_SOLVE_MIXED) {
    set_error("tn_stokes_solve_batch: modes TN_SOLVE_F64 and TN_SOLVE_F64_PREC32 only");
    return TN_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    const tn_status s = solve_check("tn_stokes_solve_batch", meshes[i], o, f[i], u[i], p[i]);
    if (s != TN_OK) return s;
    for (int k = 0; k < i; ++k)
      if (meshes[k] == meshes[i]) {
        set_error("tn_stokes_solve_batch: a mesh appears twice");
        return TN_EINVAL;
      }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool prec32 = o.mode == TN_SOLVE_F64_PREC32;
  auto t0 = std::chrono::steady_clock::now();
  g_err = cudaSuccess;
  std::vector<LockSys> sys(n);
  std::vector<double> bnorm(n, 0.0), res(n, 0.0);
  std::vector<int> why(n, FGMRES_OK);
  std::vector<KVec<double>> bs(n);
  tn_status first = TN_OK;
  for (int i = 0; i < n; ++i) status[i] = TN_OK;
  for (int i = 0; i < n; ++i) {
    status[i] = solve_begin(meshes[i], o, f[i], g ? g[i] : nullptr, u[i], p[i], st, stream, bs[i], sys[i].x, bnorm[i]);
    LockSys& q = sys[i];
    q.mesh = meshes[i];
    q.m = meshes[i]->mg;
    q.b = bs[i];
    q.abstol = o.rtol * bnorm[i];
    res[i] = bnorm[i];
    if (status[i] != TN_OK || !std::isfinite(bnorm[i]) || !(bnorm[i] > 0)) q.phase = 2;
    if (status[i] == TN_OK && !std::isfinite(bnorm[i])) why[i] = FGMRES_NONFINITE;
    if (status[i] == TN_OK && cudaMallocHost((void**)&q.hs, sizeof(double) * S_MAX) != cudaSuccess) {
      status[i] = TN_ENOMEM;
      q.phase = 2;
    }
  }
  fgmres_lockstep(sys, o.restart, o.max_iters, prec32, st);
  for (int i = 0; i < n; ++i) {
    LockSys& q = sys[i];
    if (status[i] == TN_OK) {
      if (why[i] == FGMRES_OK) why[i] = q.why;
      if (bnorm[i] > 0 && std::isfinite(bnorm[i])) res[i] = solve_true_residual(q.mesh, q.b, q.x, st);
      ck(cudaStreamSynchronize(st));
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      status[i] = solve_status("tn_stokes_solve_batch", o, q.its, 0, why[i], res[i], bnorm[i], secs,
                               stats ? &stats[i] : nullptr);
    }
    if (q.hs) cudaFreeHost(q.hs);
    if (first == TN_OK && status[i] != TN_OK) first = status[i];
  }
  return first;
}

}  // extern "C"
