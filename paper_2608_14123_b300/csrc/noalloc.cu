// Schwarz correction with a statically allocated scratch buffer.
//
// Some callers cannot allocate device memory at the point where they need a
// smoothing step: code that runs while its own CUDA stream capture is active
// (cudaMalloc is not permitted during a global-mode capture), code inside a
// framework whose caching allocator owns the device memory and forbids side
// allocations, and real-time loops that must not allocate.  For them this
// file provides one entry point that computes a Schwarz correction without
// allocating: the weighted subdomain-correction patches live in a file-scope
// __device__ array of fixed size instead of the context's patch buffer.
#include <mutex>

#include "dgfas_internal.h"

// Maximum number of FP64 patch entries: n_elem * (p + 1 + 2 m)^3 of a level
// must not exceed this (16 MiB; e.g. 954 elements at p = 8 with two overlap
// layers, 6114 elements at p = 4).  Every GPU that loads the library holds
// the array until the process exits.
#define DGFAS_STATIC_PATCH_DOUBLES (1 << 21)

static __device__ __align__(256) double g_static_patch[DGFAS_STATIC_PATCH_DOUBLES];

int launch_fd_patch(Ctx& c, int l, const double* r, double* patch);
int launch_combine_patch(Ctx& c, int l, const double* patch, double* u);

// Device address of g_static_patch, looked up once per device (host code must
// not pass the symbol itself to a kernel: on the host it names a stand-in).
static std::mutex g_mu;
static double* g_addr[64] = {nullptr};

static int static_patch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    set_error("no current CUDA device");
    return DGFAS_ERR_CUDA;
  }
  if (dev >= 64) {
    set_error("schwarz_correct_static: device ordinals of 64 and above are not supported");
    return DGFAS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_patch);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return DGFAS_ERR_CUDA;
    }
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return DGFAS_OK;
}

extern "C" int dgfas_schwarz_correct_static(void* ctx, int level, const double* r, double* u) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !r || !u || level < 1 || level >= (int)c->lv.size()) {
    set_error("schwarz_correct_static: invalid argument");
    return DGFAS_ERR_INVALID;
  }
  LevelHost& H = c->lv[level];
  const size_t need = (size_t)H.ne * H.nsm * H.nsm * H.nsm;
  if (need > (size_t)DGFAS_STATIC_PATCH_DOUBLES) {
    set_error("schwarz_correct_static: level needs " + std::to_string(need) +
              " patch entries, the static buffer holds " +
              std::to_string(DGFAS_STATIC_PATCH_DOUBLES));
    return DGFAS_ERR_UNSUPPORTED;
  }
  double* patch = nullptr;
  int rc = static_patch_address(&patch);
  if (rc != DGFAS_OK) return rc;
  // every patch entry the combine step reads is written by the FD step of the
  // same call, so nothing in the shared buffer needs clearing
  rc = launch_fd_patch(*c, level, r, patch);
  if (rc != DGFAS_OK) return rc;
  return launch_combine_patch(*c, level, patch, u);
}
