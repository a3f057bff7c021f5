// tn_apply_B_static: the divergence apply with its intermediate in a static device array.
//
// tn_apply_B keeps the fine-level divergence field (one scalar per fine node, between the
// element kernel and the restriction onto the pressure space) in scratch that the mesh
// allocates.  This variant puts that intermediate in a file-scope __device__ array compiled
// into the library instead, so the call itself needs no device allocation by anyone.
#include <mutex>
#include <string>

#include "internal.h"

namespace tn {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB, held by every GPU that loads the library

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of g_static_scratch, per device (nullptr: not set up)

// Device address of the static array on the current device.  In host code the symbol is only a
// host-side stand-in; the device address comes from cudaGetSymbolAddress, once per device, with
// that device current.
cudaError_t static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

template <typename T>
cudaError_t apply_B_static_t(const tn_mesh* m, int level, const void* const* u, void* q, void* scratch,
                             cudaStream_t st) {
  const Level& F = m->lv[level];
  const Level& C = m->lv[level + 1];
  const BC bc{m->bc_in, m->bc_out};
  T* scr = (T*)scratch;
  cudaError_t e = launch_div_fine<T>(F, bc, (const T* const*)u, scr, st);
  if (e != cudaSuccess) return e;
  const T* fin[1] = {scr};
  T* cout[1] = {(T*)q};
  return launch_restrict<T>(F, C, bc, 1, 0, fin, cout, st);
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" tn_status tn_apply_B_static(tn_mesh* mesh, int level, tn_prec prec, const void* const* u_dev,
                                       void* q_dev, void* stream) {
  if (!mesh || level < 0 || level + 1 >= (int)mesh->lv.size()) {
    set_error("tn_apply_B_static: bad mesh or level");
    return TN_EINVAL;
  }
  if (!u_dev || !u_dev[0] || !u_dev[1] || !u_dev[2] || !q_dev) {
    set_error("tn_apply_B_static: NULL vector");
    return TN_EINVAL;
  }
  for (int c = 0; c < 3; ++c)
    if (u_dev[c] == q_dev) {
      set_error("tn_apply_B_static: output aliases input");
      return TN_EINVAL;
    }
  if (prec != TN_F64 && prec != TN_F32) {
    set_error("tn_apply_B_static: unknown precision");
    return TN_EINVAL;
  }
  const size_t need = (size_t)mesh->lv[level].n_layout * (prec == TN_F64 ? sizeof(double) : sizeof(float));
  if (need > kStaticScratchBytes) {
    set_error("tn_apply_B_static: level " + std::to_string(level) + " needs " + std::to_string(need) +
              " bytes of scratch (one scalar per fine node layout entry); the static scratch holds " +
              std::to_string(kStaticScratchBytes) + " bytes");
    return TN_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != mesh->device) {
    set_error("tn_apply_B_static: the mesh's device must be current");
    return TN_EINVAL;
  }
  void* scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) {
    set_error(std::string("tn_apply_B_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return TN_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  e = prec == TN_F64 ? apply_B_static_t<double>(mesh, level, u_dev, q_dev, scratch, st)
                     : apply_B_static_t<float>(mesh, level, u_dev, q_dev, scratch, st);
  if (e != cudaSuccess) {
    set_error(std::string("tn_apply_B_static: ") + cudaGetErrorString(e));
    return TN_ECUDA;
  }
  return TN_OK;
}
