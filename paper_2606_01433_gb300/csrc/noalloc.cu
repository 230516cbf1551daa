// gdsw_apply_local_noalloc: the level-l local branch of the preconditioner (gather, the
// block-LDL^T sweeps of every part, the weighted scatter) computed without allocating any
// memory.  Its only scratch -- the concatenated local vectors that gdsw_apply_local keeps in
// a workspace allocated with the context -- lives in a fixed, file-scope device array.
//
// Who needs this: code that must not allocate device memory at solve time.  Examples are a
// service that has already handed all free device memory to its own pool, and a
// latency-critical loop that cannot let a library call cudaMalloc/cudaFree (a cudaFree also
// synchronises the whole device) in the middle of a request.
#include <mutex>
#include <new>

#include "common.h"
#include "kernels.h"

namespace gdsw {

// 4 MiB of scratch, 256-byte aligned, resident on every GPU that loads the library until
// the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device with that device current.
// (In host code the array's name is only a host-side stand-in, never a device address.)
// The cache holds until the process exits; a cudaDeviceReset unloads the module, after which
// the cached address is stale, so no call may follow a reset of the device it was made on.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// dev: the device the context was set up on, which must be the current device.
static void* noalloc_scratch_address(int dev) {
  GDSW_CHECK(dev >= 0 && dev < 64, GDSW_ERR_INVALID_ARG, "device ordinal out of range");
  int cur = -1;
  GDSW_CUDA(cudaGetDevice(&cur));
  GDSW_CHECK(cur == dev, GDSW_ERR_INVALID_ARG,
             "gdsw_apply_local_noalloc: the current device (" + std::to_string(cur) +
                 ") is not the device the context was set up on (" + std::to_string(dev) + ")");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    GDSW_CHECK(e == cudaSuccess && p != nullptr, GDSW_ERR_CUDA,
               std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

static void local_solve_into(gdsw_ctx* c, int l, const double* r, double* z, void* vec, cudaStream_t s) {
  LevelDev& L = c->ld[l];
  const int64_t nv = L.nvec;
  if (L.prec == GDSW_FP64) {
    double* v = static_cast<double*>(vec);
    launch_gather<double>(r, L.gdof, v, nv, s);
    for (int k = 0; k < L.fwd.nlaunch(); ++k)
      launch_gemv<double, double>(static_cast<const double*>(L.fac), v, v, v, L.fwd, k, L.fwd_ld[k], s);
    if (L.red.launch_tile_off.size() == 2) launch_sym_reduce<double>(v, v, L.red, L.sym_T, s);
    for (int k = 0; k < L.bwd.nlaunch(); ++k)
      launch_gemv<double, double>(static_cast<const double*>(L.fac), v, v, v, L.bwd, k, L.bwd_ld[k], s);
    launch_scatter<double>(v + nv, L.sc_ptr, L.sc_pos, L.sc_w, z, L.n, 0, s);
  } else {
    float* v = static_cast<float*>(vec);
    launch_gather<float>(r, L.gdof, v, nv, s);
    for (int k = 0; k < L.fwd.nlaunch(); ++k) {
      if (L.prec == GDSW_FP32)
        launch_gemv<float, float>(static_cast<const float*>(L.fac), v, v, v, L.fwd, k, L.fwd_ld[k], s);
      else
        launch_gemv<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(L.fac), v, v, v, L.fwd, k, L.fwd_ld[k], s);
    }
    if (L.red.launch_tile_off.size() == 2) launch_sym_reduce<float>(v, v, L.red, L.sym_T, s);
    for (int k = 0; k < L.bwd.nlaunch(); ++k) {
      if (L.prec == GDSW_FP32)
        launch_gemv<float, float>(static_cast<const float*>(L.fac), v, v, v, L.bwd, k, L.bwd_ld[k], s);
      else
        launch_gemv<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(L.fac), v, v, v, L.bwd, k, L.bwd_ld[k], s);
    }
    launch_scatter<float>(v + nv, L.sc_ptr, L.sc_pos, L.sc_w, z, L.n, 0, s);
  }
}

}  // namespace gdsw

extern "C" int gdsw_apply_local_noalloc(gdsw_ctx* c, int32_t level, const double* r, double* z) {
  using namespace gdsw;
  if (!c || c->host_only || level < 0 || level >= int(c->ld.size()) || !r || !z) return GDSW_ERR_INVALID_ARG;
  try {
    const LevelDev& L = c->ld[level];
    // the two local vectors and the partial sums of the packed symmetric blocks
    const size_t need = (size_t(2) * size_t(L.nvec) + size_t(L.npart)) * (L.prec == GDSW_FP64 ? 8 : 4);
    if (need > kNoAllocScratchBytes) {
      c->err = "gdsw_apply_local_noalloc: level " + std::to_string(level) + " needs " + std::to_string(need) +
               " bytes of local workspace, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
               "-byte scratch; use gdsw_apply_local";
      return GDSW_ERR_INVALID_ARG;
    }
    void* vec = noalloc_scratch_address(c->device);
    local_solve_into(c, level, r, z, vec, c->stream);
    return GDSW_OK;
  } catch (const gdsw::Error& e) {
    c->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return GDSW_ERR_OOM;
  } catch (...) {
    c->err = "unknown error";
    return GDSW_ERR_CUDA;
  }
}
