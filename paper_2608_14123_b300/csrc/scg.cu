// Schwarz-preconditioned inexact conjugate gradients (Alg. 6) with every
// scalar of the recurrence kept on the device.
//
// Each scalar product is one kernel: the CTAs write per-CTA partial sums, and
// the last CTA to finish (ticket counter) adds the partials in index order and
// evaluates the recurrence coefficient it feeds (beta, gamma, alpha, |r|^2).
// The kernels that follow read the coefficients from device memory, so an SCG
// block issues no host synchronization and can be captured in a CUDA graph.
// The sums are deterministic: fixed grid, fixed per-thread ranges, fixed tree
// and fixed order of the partials.
//
// Reading of the first search direction: p = z (the preconditioned residual)
// in the first step, as in the inexact PCG of Golub and Ye that the method
// adopts; the step length gamma / p.q = z.r / z.A z is then the exact line
// minimum along p.  (The printed initialization p = r, left unchanged in step
// 1, makes the SCG-smoothed V-cycle diverge on the Cartesian and perturbed
// workloads.)
//
// Exit test |r| <= r_max: once it holds, a device flag sets alpha = 0 in every
// remaining step, so u and r stay as they were when the test first held (the
// same result as leaving the loop); the step count of a block is fixed, which
// is what graph capture needs.
#include <type_traits>

#include "dgfas_internal.h"

namespace {

enum { S_GAMMA = 0, S_BETA = 1, S_ALPHA = 2, S_PQ = 3, S_RR = 4, S_DONE = 5, S_RMAX2 = 6,
       S_STEPS = 7 };

constexpr int kThreads = 256;

// Block-wide sums of K values per thread (fixed tree); thread 0 gets the result.
template <int K>
__device__ void block_sum(double (&v)[K], double (*sh)[kThreads]) {
  for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  for (int k = 0; k < K; ++k) v[k] = sh[k][0];
}

// Writes this CTA's K partial sums to part[k * G + cta] and takes a ticket;
// returns true in the last CTA, which then holds the totals (partials added in
// CTA order by a fixed tree) in tot[] on every thread.
template <int K>
__device__ bool partials_and_ticket(double (&v)[K], double* part, int* counter,
                                    double (&tot)[K]) {
  __shared__ double sh[K][kThreads];
  __shared__ int last;
  block_sum<K>(v, sh);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) part[k * G + blockIdx.x] = v[k];
    __threadfence();
    last = atomicAdd(counter, 1) == G - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[K];
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  for (int i = threadIdx.x; i < G; i += kThreads)
    for (int k = 0; k < K; ++k) s[k] += __ldcg(part + k * G + i);
  block_sum<K>(s, sh);
  for (int k = 0; k < K; ++k) tot[k] = s[k];
  if (threadIdx.x == 0) *counter = 0;   // ready for the next reduction
  return true;
}

// Per-thread sum of products in the vectors' precision: FP64 for FP64
// vectors; for FP32 vectors a compensated (Kahan) FP32 sum, widened to FP64
// once per thread - B300's FP64 rate is 1/62 of its FP32 rate, so FP64
// products per element would bound these streaming kernels.
template <typename T>
struct Acc {
  double s = 0.0;
  __device__ __forceinline__ void add(T a, T b) { s += (double)a * (double)b; }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float y = __fmaf_rn(a, b, -c);
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// |r|^2 of the start residual: r_max^2 = rtol^2 |r|^2, done = (r == 0), steps = 0
template <typename T>
__global__ void k_scg_init(const T* __restrict__ r, long long n, double rtol2, double* part,
                           int* counter, double* scal) {
  Acc<T> a0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kThreads)
    a0.add(r[i], r[i]);
  double v[1] = {a0.get()};
  double t[1];
  if (partials_and_ticket<1>(v, part, counter, t) && threadIdx.x == 0) {
    scal[S_RR] = t[0];
    scal[S_RMAX2] = rtol2 * t[0];
    scal[S_DONE] = t[0] > 0.0 ? 0.0 : 1.0;
    scal[S_STEPS] = 0.0;
  }
}

// no exit test (rtol = 0): the scalars start from "not done", no reduction
// (a zero residual then gives gamma = p.q = 0 and alpha = 0, so nothing moves)
__global__ void k_scg_reset(double* scal) {
  if (threadIdx.x == 0) {
    scal[S_RMAX2] = 0.0;
    scal[S_DONE] = 0.0;
    scal[S_STEPS] = 0.0;
  }
}

// gamma_new = z.r; for step > 1 also z.r0 and beta = (z.r - z.r0) / gamma_old
// (products and sums in FP64)
template <typename T, bool FIRST>
__global__ void k_scg_zr(const T* __restrict__ z, const T* __restrict__ r,
                         const T* __restrict__ r0, long long n, double* part, int* counter,
                         double* scal) {
  Acc<T> a0, a1;
  const long long S = (long long)gridDim.x * kThreads;
  long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  // four independent strided elements per iteration keep more loads in flight
  for (; i + 3 * S < n; i += 4 * S) {
    T zz[4], rr[4], qq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zz[u] = z[i + u * S];
      rr[u] = r[i + u * S];
      if (!FIRST) qq[u] = r0[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0.add(zz[u], rr[u]);
      if (!FIRST) a1.add(zz[u], qq[u]);
    }
  }
  for (; i < n; i += S) {
    a0.add(z[i], r[i]);
    if (!FIRST) a1.add(z[i], r0[i]);
  }
  double v[2] = {a0.get(), a1.get()};
  double t[2];
  if (partials_and_ticket<2>(v, part, counter, t) && threadIdx.x == 0) {
    const bool done = scal[S_DONE] != 0.0;
    if (!FIRST) scal[S_BETA] = done ? 0.0 : (t[0] - t[1]) / scal[S_GAMMA];
    scal[S_GAMMA] = t[0];
  }
}

// p = z (first step) or p = beta p + z
template <typename T, bool FIRST>
__global__ void k_scg_dir(T* __restrict__ p, const T* __restrict__ z, long long n,
                          const double* __restrict__ scal) {
  const T beta = FIRST ? T(0) : (T)scal[S_BETA];
  const long long S = (long long)gridDim.x * kThreads;
  long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    T zz[4], pp[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zz[u] = z[i + u * S];
      if (!FIRST) pp[u] = p[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) p[i + u * S] = FIRST ? zz[u] : beta * pp[u] + zz[u];
  }
  for (; i < n; i += S) p[i] = FIRST ? z[i] : beta * p[i] + z[i];
}

// pq = p.q, alpha = gamma / pq (0 once the exit test held, or for pq = 0)
template <typename T>
__global__ void k_scg_pq(const T* __restrict__ p, const T* __restrict__ q, long long n,
                         double* part, int* counter, double* scal) {
  Acc<T> a0;
  const long long S = (long long)gridDim.x * kThreads;
  long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    T pp[4], qq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pp[u] = p[i + u * S];
      qq[u] = q[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) a0.add(pp[u], qq[u]);
  }
  for (; i < n; i += S) a0.add(p[i], q[i]);
  double v[1] = {a0.get()};
  double t[1];
  if (partials_and_ticket<1>(v, part, counter, t) && threadIdx.x == 0) {
    scal[S_PQ] = t[0];
    const bool done = scal[S_DONE] != 0.0;
    scal[S_ALPHA] = (done || t[0] == 0.0) ? 0.0 : scal[S_GAMMA] / t[0];
  }
}

// r0 = r; r -= alpha q; x += alpha p; |r|^2 and the exit test |r| <= r_max.
// With uout (the last step of a correction-form block, no exit test):
// uout += x + alpha p instead of storing x.
template <typename T>
__global__ void k_scg_update(T* __restrict__ r, T* __restrict__ r0, T* __restrict__ x,
                             const T* __restrict__ p, const T* __restrict__ q, long long n,
                             double* part, int* counter, double* scal, double* __restrict__ uout) {
  const T alpha = (T)scal[S_ALPHA];
  Acc<T> a0;
  const long long S = (long long)gridDim.x * kThreads;
  long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    T rr[4], qq[4], xx[4], pp[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rr[u] = r[i + u * S];
      qq[u] = q[i + u * S];
      xx[u] = x[i + u * S];
      pp[u] = p[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const T rn = rr[u] - alpha * qq[u];
      r0[i + u * S] = rr[u];
      r[i + u * S] = rn;
      const T xn = xx[u] + alpha * pp[u];
      if (uout) uout[i + u * S] += (double)xn;
      else x[i + u * S] = xn;
      a0.add(rn, rn);
    }
  }
  for (; i < n; i += S) {
    const T ri = r[i];
    const T rn = ri - alpha * q[i];
    r0[i] = ri;
    r[i] = rn;
    const T xn = x[i] + alpha * p[i];
    if (uout) uout[i] += (double)xn;
    else x[i] = xn;
    a0.add(rn, rn);
  }
  double v[1] = {a0.get()};
  double t[1];
  if (partials_and_ticket<1>(v, part, counter, t) && threadIdx.x == 0) {
    if (scal[S_DONE] == 0.0) {
      scal[S_RR] = t[0];
      scal[S_STEPS] += 1.0;
      if (t[0] <= scal[S_RMAX2]) scal[S_DONE] = 1.0;
    }
  }
}

// y = (double) x
__global__ void k_scg_to_double(const float* __restrict__ x, double* __restrict__ y, long long n) {
  const long long S = (long long)gridDim.x * kThreads;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += S)
    y[i] = (double)x[i];
}

}  // namespace

#define LAUNCH_CHECK()                                      \
  do {                                                      \
    ++g_kernels;                                            \
    if (cudaGetLastError() != cudaSuccess) {                \
      set_error("scg kernel launch");                       \
      return DGFAS_ERR_CUDA;                                \
    }                                                       \
  } while (0)

// The Schwarz sweep z = sum_e R^T W A~^-1 R r of SCG in precision prec, and the
// operator q = A p in the vectors' precision T.
static int scg_sweep(Ctx& c, int l, int prec, const double* r, double* z) {
  const long long nd = c.lv[l].ndof;
  if (prec == DGFAS_FP64) {
    if (cudaMemcpyAsync(c.rw, r, nd * sizeof(double), cudaMemcpyDeviceToDevice, c.stream) !=
        cudaSuccess) {
      set_error("scg: copy");
      return DGFAS_ERR_CUDA;
    }
  } else {
    int rc = launch_to_float(c, r, (float*)c.rw, nd);
    if (rc != DGFAS_OK) return rc;
  }
  int rc = launch_fd(c, l, prec, c.rw);
  return rc == DGFAS_OK ? launch_combine_to(c, l, prec, z) : rc;
}
static int scg_sweep(Ctx& c, int l, int prec, const float* r, float* z) {
  int rc = launch_fd(c, l, prec, r);
  return rc == DGFAS_OK ? launch_combine_to32(c, l, z) : rc;
}
static int scg_apply(Ctx& c, int l, const double* p, double* q) {
  return launch_apply(c, l, DGFAS_FP64, p, nullptr, q, 1.0);
}
static int scg_apply(Ctx& c, int l, const float* p, float* q) { return launch_apply32(c, l, p, q); }

// n steps of Alg. 6 on A x = b given the start residual r = b - A x; x and r
// updated in place; p, q, z, r0 work vectors of the level's size.
template <typename T>
static int scg_steps(Ctx& c, int l, int prec, T* x, T* r, T* p, T* q, T* z, T* r0, int n,
                     double rtol, double* uout = nullptr) {
  const long long nd = c.lv[l].ndof;
  double* scal = c.dscal;
  int* cnt = c.dcnt;
  // 8 CTAs of 256 threads per SM for the streaming kernels; their partial
  // sums (two per CTA at most) live past the first red_blocks entries of the
  // reduction buffer, which hold the cycle's residual norm partials until the
  // host reads them
  const int G = 2 * c.red_blocks;
  double* part = c.red + c.red_blocks;
  if (rtol > 0.0) {
    k_scg_init<T><<<G, kThreads, 0, c.stream>>>(r, nd, rtol * rtol, part, cnt, scal);
  } else {
    k_scg_reset<<<1, 32, 0, c.stream>>>(scal);
  }
  LAUNCH_CHECK();
  for (int i = 1; i <= n; ++i) {
    int rc = scg_sweep(c, l, prec, r, z);
    if (rc != DGFAS_OK) return rc;
    if (i == 1) {
      k_scg_zr<T, true><<<G, kThreads, 0, c.stream>>>(z, r, nullptr, nd, part, cnt, scal);
      LAUNCH_CHECK();
      k_scg_dir<T, true><<<G, kThreads, 0, c.stream>>>(p, z, nd, scal);
      LAUNCH_CHECK();
    } else {
      k_scg_zr<T, false><<<G, kThreads, 0, c.stream>>>(z, r, r0, nd, part, cnt, scal);
      LAUNCH_CHECK();
      k_scg_dir<T, false><<<G, kThreads, 0, c.stream>>>(p, z, nd, scal);
      LAUNCH_CHECK();
    }
    rc = scg_apply(c, l, p, q);
    if (rc != DGFAS_OK) return rc;
    k_scg_pq<T><<<G, kThreads, 0, c.stream>>>(p, q, nd, part, cnt, scal);
    LAUNCH_CHECK();
    k_scg_update<T><<<G, kThreads, 0, c.stream>>>(r, r0, x, p, q, nd, part, cnt, scal,
                                                   i == n ? uout : nullptr);
    LAUNCH_CHECK();
  }
  return DGFAS_OK;
}

// Alg. 6 on level l with n steps from the FP64 residual in lv[l].r (= g - A u),
// u updated in place; rtol > 0 adds the exit test |r| <= rtol |r_start|.  No
// host synchronization.
// prec = FP64: the iteration itself, in FP64; lv[l].r ends as the CG residual
// (want_res is the caller's business).
// prec = FP32 / BF16: correction form, as the WAS smoother: SCG on A d = r in
// FP32 vectors (FP32 operator, Schwarz sweep in prec, FP64 scalar products),
// then u += d.  In exact arithmetic the iterates are the same; the FP64
// residual of the outer cycle drives the iterative refinement.  d starts at
// zero, or with `pending` at the correction already in lv[l].delta (the
// prolongation, not yet in u; lv[l].r is then the residual of u without it),
// the start residual r - A d being formed in the smoother precision.  With
// want_res, lv[l].r becomes SCG's recursive residual r - A d (FP32, widened
// to FP64), the residual of the new u in the smoother precision; otherwise
// lv[l].r is stale afterwards.
// fp64_vectors: FP64 iteration (vectors, operator, recurrences) whatever
// prec is; prec then only sets the precision of the Schwarz sweep (the
// preconditioner), as for the root solve in a mixed-precision context.
int scg_run(Ctx& c, int l, double* u, int n, double rtol, int prec, bool pending,
            bool want_res, bool fp64_vectors) {
  LevelHost& H = c.lv[l];
  const long long nd = H.ndof;
  if (!c.scg_buf) {
    set_error("scg: no SCG work vectors (context not set up for SCG)");
    return DGFAS_ERR_INVALID;
  }
  // consecutive work vectors are staggered by a few KB (kScgPad doubles) so
  // that the same index of the streams does not fall at the same offset of a
  // large power of two (the vectors of a big level are 2^29 bytes long)
  if (prec == DGFAS_FP64 || fp64_vectors) {
    if (pending) {
      set_error("scg: a pending correction needs the smoother-precision path");
      return DGFAS_ERR_INVALID;
    }
    const long long s = nd + kScgPad;
    double *p = c.scg_buf, *q = p + s, *z = q + s, *r0 = z + s;
    return scg_steps<double>(c, l, prec, u, H.r, p, q, z, r0, n, rtol);
  }
  float* d = (float*)H.delta;
  const long long s = nd + 2 * kScgPad;
  float *r = (float*)c.scg_buf, *p = r + s, *q = p + s, *z = q + s, *r0 = z + s;
  int rc = DGFAS_OK;
  if (pending) {
    rc = launch_apply_corr(c, l, prec, d, H.r, r, 0);   // r = r_u - A d
  } else {
    if (cudaMemsetAsync(d, 0, nd * sizeof(float), c.stream) != cudaSuccess) {
      set_error("scg: memset");
      return DGFAS_ERR_CUDA;
    }
    rc = launch_to_float(c, H.r, r, nd);
  }
  // without an exit test the last step adds the correction to u directly
  const bool fuse = n > 0 && !(rtol > 0.0);
  if (rc == DGFAS_OK) rc = scg_steps<float>(c, l, prec, d, r, p, q, z, r0, n, rtol,
                                            fuse ? u : nullptr);
  if (rc == DGFAS_OK && want_res) {
    // the residual of the new u: SCG's recursive residual r_start - A d
    k_scg_to_double<<<c.red_blocks, kThreads, 0, c.stream>>>(r, H.r, nd);
    LAUNCH_CHECK();
  }
  if (rc == DGFAS_OK && !fuse) rc = launch_add_delta(c, nd, prec, d, u);
  return rc;
}

// Outcome of the last SCG block on the context's stream (synchronizes):
// out[0] = |r|^2 when its exit test last ran (or at the start), out[1] = steps
// taken before the exit test held (all steps if it never did), out[2] = 1 if
// the exit test |r| <= rtol |r_start| held, else 0.
extern "C" int dgfas_scg_info(void* ctx, double* out_host) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out_host) return DGFAS_ERR_INVALID;
  double s[8];
  if (cudaMemcpyAsync(s, c->dscal, sizeof(s), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    set_error("scg_info: copy");
    return DGFAS_ERR_CUDA;
  }
  out_host[0] = s[S_RR];
  out_host[1] = s[S_STEPS];
  out_host[2] = s[S_DONE];
  return DGFAS_OK;
}

// Per-kernel timing of one SCG step on `level` in the context's smoother
// precision, with CUDA events on the context's stream, averaged over `reps`
// steps from the residual g - A u: ms_out[0..5] = the FD kernel of the Schwarz
// sweep, its combine, the scalar product z.r (with beta) and the direction
// update, the operator q = A p, the scalar product p.q and the fused
// residual / iterate update, and the FP64 residual apply of the V-cycle.
// Level vectors are scratch afterwards; u is not modified.
extern "C" int dgfas_profile_scg(void* ctx, int level, double* u, const double* g, int reps,
                                 double* ms_out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !g || !ms_out || reps <= 0 || level < 1 || level >= (int)c->lv.size() ||
      !c->scg_buf)
    return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  const long long nd = H.ndof;
  const int prec = c->prm.precision;
  const int G = 2 * c->red_blocks;
  double* part = c->red + c->red_blocks;
  cudaEvent_t ev[7];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return DGFAS_ERR_CUDA;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int rc = launch_apply(*c, level, DGFAS_FP64, u, g, H.r, -1.0);
  auto step = [&](auto* x, auto* r, auto* p, auto* q, auto* z, auto* r0) -> int {
    using T = std::remove_pointer_t<decltype(x)>;
    int e = DGFAS_OK;
    k_scg_init<T><<<G, kThreads, 0, c->stream>>>(r, nd, 0.0, part, c->dcnt, c->dscal);
    for (int it = 0; it < reps && e == DGFAS_OK; ++it) {
      cudaEventRecord(ev[0], c->stream);
      if constexpr (sizeof(T) == 8) {
        cudaMemcpyAsync(c->rw, r, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        e = launch_fd(*c, level, prec, c->rw);
        cudaEventRecord(ev[1], c->stream);
        if (e == DGFAS_OK) e = launch_combine_to(*c, level, prec, (double*)z);
      } else {
        e = launch_fd(*c, level, prec, r);
        cudaEventRecord(ev[1], c->stream);
        if (e == DGFAS_OK) e = launch_combine_to32(*c, level, (float*)z);
      }
      cudaEventRecord(ev[2], c->stream);
      k_scg_zr<T, false><<<G, kThreads, 0, c->stream>>>(z, r, r0, nd, part, c->dcnt, c->dscal);
      k_scg_dir<T, false><<<G, kThreads, 0, c->stream>>>(p, z, nd, c->dscal);
      cudaEventRecord(ev[3], c->stream);
      if (e == DGFAS_OK) e = scg_apply(*c, level, p, q);
      cudaEventRecord(ev[4], c->stream);
      k_scg_pq<T><<<G, kThreads, 0, c->stream>>>(p, q, nd, part, c->dcnt, c->dscal);
      k_scg_update<T><<<G, kThreads, 0, c->stream>>>(r, r0, x, p, q, nd, part, c->dcnt, c->dscal,
                                                      nullptr);
      cudaEventRecord(ev[5], c->stream);
      if (e == DGFAS_OK) e = launch_apply(*c, level, DGFAS_FP64, u, g, H.t ? H.t : H.r, -1.0);
      cudaEventRecord(ev[6], c->stream);
      if (cudaEventSynchronize(ev[6]) != cudaSuccess) e = DGFAS_ERR_CUDA;
      for (int k = 0; k < 6 && e == DGFAS_OK; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        acc[k] += ms;
      }
    }
    return e;
  };
  if (rc == DGFAS_OK) {
    if (prec == DGFAS_FP64) {
      const long long s = nd + kScgPad;
      double *p = c->scg_buf, *q = p + s, *z = q + s, *r0 = z + s;
      cudaMemcpyAsync(r0, H.r, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(p, H.r, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(H.delta, u, nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      // the iterate is a copy of u (in the level's FP64 correction buffer), so
      // u stays as it was
      rc = step((double*)H.delta, H.r, p, q, z, r0);
    } else {
      const long long s = nd + 2 * kScgPad;
      float *r = (float*)c->scg_buf, *p = r + s, *q = p + s, *z = q + s, *r0 = z + s;
      cudaMemsetAsync(H.delta, 0, nd * sizeof(float), c->stream);
      rc = launch_to_float(*c, H.r, r, nd);
      cudaMemcpyAsync(r0, r, nd * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(p, r, nd * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
      if (rc == DGFAS_OK) rc = step((float*)H.delta, r, p, q, z, r0);
    }
  }
  if (rc == DGFAS_OK && cudaGetLastError() != cudaSuccess) rc = DGFAS_ERR_CUDA;
  for (int k = 0; k < 6; ++k) ms_out[k] = acc[k] / reps;
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}
