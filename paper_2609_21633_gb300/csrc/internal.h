// Internal definitions shared by the host mesh code, the kernels and the C ABI.
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/terra_wedge.h"

namespace tn {

constexpr int kLayerStride = 12;  // values per radial cell in the layer table
constexpr int kDiagCoef = 24;     // values per lateral triangle in the diag(A) factor table

// Per-level mesh data.  Host vectors hold the definition; device pointers are
// owned by the level and freed by tn_mesh_destroy.
struct Level {
  int l = 0, N = 0, n_r = 0, P = 0;  // lateral level, 2^l, node layers, row pitch
  int64_t layer_stride = 0, diamond_stride = 0, n_layout = 0;
  int64_t n_tri = 0, n_wedges = 0, n_lat_layout = 0;  // 10 N^2 2, n_tri (n_r-1), 10 (N+1) P

  std::vector<double> lat_xyz;  // (10, N+1, N+1, 3)
  std::vector<double> radii;    // n_r

  // Geometry per lateral triangle t = ((d N + i) N + j) 2 + w, SoA over q:
  // q = 0..8: M^{-1}[m][x] (row-major), q = 9: |det M|, M = [s1 - s0, s2 - s0, (s0+s1+s2)/3].
  double* geo64 = nullptr;
  float* geo32 = nullptr;
  // Per radial cell k (kLayerStride values): w0 = 1/(2 rho), w1 = 1/(6 h), vol = rho^2 h, rho,
  // w1 / w0, vol w0^2, vol w0, -vol w0 / 6, w0 / (9 w1), vol w1^2, 0, 0;
  // rho = (r_k + r_k+1)/2, h = (r_k+1 - r_k)/2.
  double* lay64 = nullptr;
  float* lay32 = nullptr;
  // The same table as double-float pairs (hi, lo) for the double-float element ops (df = 1).
  float* laydf = nullptr;
  int df = 0;
  // Lateral unit vectors s, SoA [3][10 (N+1) P] in lateral layout (d (N+1) + i) P + j.
  double* s64 = nullptr;
  float* s32 = nullptr;
  // Interface groups: lattice points shared by several diamonds.
  int n_groups = 0;
  int* grp_ptr = nullptr;       // n_groups + 1
  int64_t* grp_off = nullptr;   // copy offsets d * diamond_stride + i * P + j, ascending per group
  double* grp_s64 = nullptr;    // [3][n_groups] unit vector of the group's point
  float* grp_s32 = nullptr;
  uint8_t* owned = nullptr;     // [10 (N+1) P] 1 if this copy is the canonical one (or not shared)
  std::vector<int> h_grp_ptr;
  std::vector<int64_t> h_grp_off;
  // Viscosity per wedge (wedge layout).  The FP32 kernels read eta32 (eta_kind 0) or the 16-bit
  // eta16 (eta_kind = TN_ETA_BF16 / TN_ETA_F16) times eta_cs[t], one factor per lateral wedge
  // t = ((d N + i) N + j) 2 + w (its radial column).
  double* eta64 = nullptr;
  float* eta32 = nullptr;
  int eta_kind = TN_ETA_F32;
  // Hourglass control of the A block (0: off): eps_e = hg_kappa tr(A_e) / 18.
  double hg_kappa = 0;
  // Radial quadrature points of the A block (1: the barycentre; 2: two-point Gauss in zeta).
  int quad = 1;
  // Per-triangle factors of the diagonal of A ([24][n_tri], see OpDiag), for div term dcoef_div.
  double* dcoef64 = nullptr;
  float* dcoef32 = nullptr;
  float* dcoefdf = nullptr;  // the same table as double-float pairs (hi, lo)
  // ... and per cell (the two triangles t = 2 p, 2 p + 1 of a lateral cell): [q][n_tri / 2] float4
  // (hi of t, hi of t + 1, lo of t, lo of t + 1), the lanes of the packed double-float diagonal
  float4* dcoefdf2 = nullptr;
  int dcoef_div = -1;
  // Tile-line partial sums of the FP64 halo-free tile kernels (levels with N >= 32):
  // [4 slots][3 components][n_r][10][tile-line nodes of a diamond layer]; the FP32 paired-cell
  // tiles use the same allocation as float4 entries [4 slots][n_r][10][tile-line nodes].
  double* ring64 = nullptr;
  // (diamond, i, j, 0) of every interface copy (grp_off order), levels with a ring buffer.
  int4* grp_dij = nullptr;
  uint16_t* eta16 = nullptr;
  float* eta_cs = nullptr;
  // Scratch scalar field in this level's node layout (B / B^T intermediate).
  double* scr64 = nullptr;
  float* scr32 = nullptr;
  // Weight mask over the node layout: 1 on the canonical copy of every node, 0 on other
  // copies and on padding (Euclidean inner products over unique nodes).
  uint8_t* wmask = nullptr;
  // TALA reference state (tn_set_reference_state; level 0 only): tala = 1 when set, the layer
  // tables then carry rho(q_c) in slot 10 and rho'(q_c) / (6 w0) in slot 11; bw64 is the buoyancy
  // weight rho(q_c) alpha(q_c) per radial cell (n_r - 1 values, nullptr = Boussinesq).
  int tala = 0;
  double* bw64 = nullptr;
  std::vector<double> h_lay;  // host copy of the layer table
  // Unit radial direction r_hat(q_c) = sbar / |sbar| per lateral triangle, SoA [3][n_tri] (FP64,
  // FP32 and double-float pairs): the TALA divergence's rho' term.
  double* rhat64 = nullptr;
  float* rhat32 = nullptr;
  float* rhatdf = nullptr;
  double* rad64 = nullptr;  // node radii r_k
  float* rad32 = nullptr;
  double inertia[3][3] = {};  // sum over unique nodes of |x|^2 I - x x^T (rotation Gram matrix)
};

// Index sizes handed to kernels.
struct Dims {
  int N, n_r, P;
  int64_t layer_stride, diamond_stride, n_tri, n_lat_layout;
};
inline Dims dims(const Level& L) {
  return Dims{L.N, L.n_r, L.P, L.layer_stride, L.diamond_stride, L.n_tri, L.n_lat_layout};
}

}  // namespace tn

namespace tn {
struct MGState;
void mg_free(MGState*);
}

namespace tn {
// Energy-equation workspace of a mesh (level 0): lumped mass, four work vectors, a reduction
// buffer and the cached largest eigenvalue of M^-1 K (0: not computed); freed by energy_free.
struct EnergyState {
  double* mass = nullptr;
  double* w[4] = {};
  double* part = nullptr;
  double lambda = 0;
};
}  // namespace tn

struct tn_mesh {
  std::vector<tn::Level> lv;
  tn::MGState* mg = nullptr;
  int bc_in = TN_BC_FREESLIP, bc_out = TN_BC_FREESLIP, div_term = 1;
  bool eta_set = false;
  int eta_storage = TN_ETA_F32;
  double hg_kappa = 0;
  int quad = 1;
  int df = 1;  // FP64 A element arithmetic in double-float (tn_mesh_opts.fp64_element)
  int device = 0;
  double r_in = 0, r_out = 0;
  // Device buffers of tn_operator_steps_host: two sets of the step's 14 vectors (u 3, p, y_A 3,
  // q, y_BT 3, d 3), element size hs_elem (0: not allocated).
  void* hs_buf[2][14] = {};
  size_t hs_elem = 0;
  // Cancel flag that tn_stokes_solve polls once per Krylov iteration (set by the server's
  // tn_server_cancel; nullptr: never cancelled).
  std::atomic<int>* cancel = nullptr;
  tn::EnergyState en;
};

namespace tn {

// Host mesh construction (mesh.cpp).
void build_lateral_points(int level, std::vector<double>& pts);
void build_level_host(Level& L, int level, int n_r, double r_in, double r_out, std::vector<double>& geo,
                      std::vector<double>& lay, std::vector<double>& s, std::vector<int>& grp_ptr,
                      std::vector<int64_t>& grp_off, std::vector<double>& grp_s, std::vector<uint8_t>& owned,
                      std::string& err);

void set_error(const std::string& msg);
void energy_free(tn_mesh* mesh);
// Tables and device arrays of one level (api.cu); destroy_level frees them.
tn_status create_level(Level& L, int l, int nr, double r_in, double r_out, int eta_storage, int div_term);
void destroy_level(Level& L);
void mg_invalidate(tn_mesh* mesh);

// ---- kernel launchers (kernels.cu) --------------------------------------------------------
struct BC {
  int in, out;  // TN_BC_* at node layer 0 and n_r - 1
};
template <typename T>
cudaError_t launch_apply_A(const Level& L, BC bc, int div_term, const T* const* u, T* const* y, cudaStream_t st,
                           const int* skip = nullptr);

// Vector updates fused into the epilogue of the A apply (y = K x, never stored except as a
// partial sum at diamond-edge nodes):
//   EPI_RESID: r = b - y
//   EPI_CHEB1: r = b - y, d_out = c0 D^-1 r, x_out = x + d_out           (x = the apply input)
//   EPI_CHEB2: r = r - y, d_out = c1 d + c2 D^-1 r, x_out = x_acc + d_out  (d = the apply input)
// D^-1 = inverse 3x3 node blocks (xx, yy, zz, xy, xz, yz).  Outputs must not alias the inputs
// the apply reads (x or d); r and x_acc / x_out may be updated in place.
enum { EPI_NONE = 0, EPI_RESID = 1, EPI_CHEB1 = 2, EPI_CHEB2 = 3 };
template <typename T>
struct EpiArgs {
  const T* b[3];
  T* r[3];
  const T* binv[6];
  const T* xacc[3];  // CHEB2: x before the update
  T* dout[3];
  T* xout[3];
  double c0, c1, c2;
};
template <typename T>
cudaError_t launch_apply_A_epi(const Level& L, BC bc, int div_term, int epi, const T* const* in, const EpiArgs<T>& E,
                               T* const* t, cudaStream_t st, const int* skip = nullptr);
template <typename T>
cudaError_t launch_div_fine(const Level& L, BC bc, const T* const* u, T* q, cudaStream_t st);
template <typename T>
cudaError_t launch_grad_fine(const Level& L, BC bc, const T* p, T* const* y, cudaStream_t st);
template <typename T>
cudaError_t launch_diag_A(const Level& L, BC bc, int div_term, T* const* d, cudaStream_t st);
// Inverse of the 3x3 node blocks of P A P + I - P (6 arrays: xx, yy, zz, xy, xz, yz).
template <typename T>
cudaError_t launch_block_inv_A(const Level& L, BC bc, int div_term, T* const* b, cudaStream_t st);
template <typename T>
cudaError_t launch_diag_pmass(const Level& F, const Level& C, T* m, cudaStream_t st);
// Interface sum over shared copies; mode 0: plain sum; 1: + (I - P) u at boundary layers;
// 2: + diag(I - P) at boundary layers.
template <typename T>
cudaError_t launch_interface(const Level& L, BC bc, int ncomp, int mode, T* const* y, const T* const* u,
                             cudaStream_t st, const int* skip = nullptr);
template <typename T>
cudaError_t launch_prolong(const Level& F, const Level& C, BC bc, int ncomp, int apply_bc, const T* const* c,
                           T* const* f, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const Level& F, const Level& C, BC bc, int ncomp, int apply_bc, const T* const* f,
                            T* const* c, cudaStream_t st);
cudaError_t launch_eta_from_T(const Level& L, const double* T, double E, double jump_r, double jump_f, double* eta,
                              cudaStream_t st);
cudaError_t launch_eta_coarsen(const Level& F, const Level& C, const double* ef, double* ec, cudaStream_t st);
cudaError_t launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t st);
// Kernel attributes that must be set before the first launch (shared-memory opt-ins); called
// once per process by tn_mesh_create.
cudaError_t prepare_tile_kernels();
// Entries of Level::ring64 for a level (0: the level needs none).
int64_t ring_buffer_entries(int N, int n_r);
// The FP32 path's viscosity from eta64: eta32, or eta16 and the column factors (see Level).
cudaError_t launch_eta_f32_path(const Level& L, cudaStream_t st);
cudaError_t launch_buoyancy(const Level& L, BC bc, const double* T, double Ra, double* const* f, cudaStream_t st);
// Energy equation (Eq. energy): residual R = (K + C(u) + S(u)) T (u NULL: diffusion only; supg: the
// streamline-upwind term) and the lumped mass, FP64, with the interface sum (energy.cu drives them).
cudaError_t launch_energy_residual(const Level& L, const double* const* u, const double* T, double* R, int supg,
                                   cudaStream_t st);
cudaError_t launch_lumped_mass(const Level& L, double* m, cudaStream_t st);

}  // namespace tn
