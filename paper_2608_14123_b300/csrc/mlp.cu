// Learned tensor-product surrogate: a 24 -> 64 -> 64 -> 6 MLP (tanh hidden,
// linear output, FP32) mapping an element's normalized corner coordinates to
// (log dx_i / V^(1/3), log s_i), i = 1..3, from which the coefficients of the
// surrogate operator of Eq. (10) are g_i = s_i nu dx_j dx_k / (2 dx_i).
// Hand-written training (forward, backward, Adam) and inference kernels.
// Parameter layout (flat, row-major): W1[64][24] b1[64] W2[64][64] b2[64]
// W3[6][64] b3[6].
#include <atomic>
#include <cmath>
#include <vector>

#include "dgfas_internal.h"

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
      return DGFAS_ERR_CUDA;                                                  \
    }                                                                         \
  } while (0)
#define RET(x)                       \
  do {                               \
    int rc_ = (x);                   \
    if (rc_ != DGFAS_OK) return rc_; \
  } while (0)

static const int H0 = 24, H1 = 64, H2 = 64, H3 = 6;
static const int OFF_W1 = 0, OFF_B1 = OFF_W1 + H1 * H0, OFF_W2 = OFF_B1 + H1,
                 OFF_B2 = OFF_W2 + H2 * H1, OFF_W3 = OFF_B2 + H2, OFF_B3 = OFF_W3 + H3 * H2,
                 NPARAM = OFF_B3 + H3;

// y[n][o] = act(sum_i W[o][i] x[n][i] + b[o]); thread per (n, o)
template <bool TANH>
__global__ void k_dense_fwd(const float* __restrict__ W, const float* __restrict__ b,
                            const float* __restrict__ x, float* __restrict__ y, int n, int nin,
                            int nout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nout) return;
  const int s = t / nout, o = t % nout;
  float z = b[o];
  for (int i = 0; i < nin; ++i) z = fmaf(W[o * nin + i], x[s * nin + i], z);
  y[t] = TANH ? tanhf(z) : z;
}

// output delta of the MSE loss: d[n][o] = 2 (y - t) / (n * nout)
__global__ void k_out_delta(const float* __restrict__ y, const float* __restrict__ tgt,
                            float* __restrict__ d, int n, int nout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nout) return;
  d[t] = 2.0f * (y[t] - tgt[t]) / (float)(n * nout);
}

// previous-layer delta through a tanh layer: dp[n][i] = (sum_o d[n][o] W[o][i]) (1 - a[n][i]^2)
__global__ void k_back_delta(const float* __restrict__ W, const float* __restrict__ d,
                             const float* __restrict__ a, float* __restrict__ dp, int n, int nin,
                             int nout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nin) return;
  const int s = t / nin, i = t % nin;
  float acc = 0.0f;
  for (int o = 0; o < nout; ++o) acc = fmaf(d[s * nout + o], W[o * nin + i], acc);
  const float ai = a[t];
  dp[t] = acc * (1.0f - ai * ai);
}

// weight and bias gradients: gW[o][i] = sum_n d[n][o] x[n][i], gb[o] = sum_n d[n][o]
// (one thread per entry, samples summed in order: deterministic)
__global__ void k_wgrad(const float* __restrict__ d, const float* __restrict__ x,
                        float* __restrict__ gW, float* __restrict__ gb, int n, int nin,
                        int nout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nout * nin) {
    const int o = t / nin, i = t % nin;
    float acc = 0.0f;
    for (int s = 0; s < n; ++s) acc = fmaf(d[s * nout + o], x[s * nin + i], acc);
    gW[t] = acc;
  } else if (t < nout * nin + nout) {
    const int o = t - nout * nin;
    float acc = 0.0f;
    for (int s = 0; s < n; ++s) acc += d[s * nout + o];
    gb[o] = acc;
  }
}

// Adam with bias correction (step t >= 1)
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int np, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const float gi = g[t];
  const float mi = b1 * m[t] + (1.0f - b1) * gi;
  const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
  m[t] = mi;
  v[t] = vi;
  th[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ idx,
                              float* __restrict__ dst, int n, int w) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * w) return;
  dst[t] = src[(size_t)idx[t / w] * w + t % w];
}

static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

struct MlpWork {
  float *a1, *a2, *y, *d3, *d2, *d1;
};

static int mlp_forward_dev(cudaStream_t st, const float* th, const float* X, int n, MlpWork& w) {
  k_dense_fwd<true><<<nb((long long)n * H1), 256, 0, st>>>(th + OFF_W1, th + OFF_B1, X, w.a1, n, H0, H1);
  k_dense_fwd<true><<<nb((long long)n * H2), 256, 0, st>>>(th + OFF_W2, th + OFF_B2, w.a1, w.a2, n, H1, H2);
  k_dense_fwd<false><<<nb((long long)n * H3), 256, 0, st>>>(th + OFF_W3, th + OFF_B3, w.a2, w.y, n, H2, H3);
  g_kernels += 3;
  CK(cudaGetLastError());
  return DGFAS_OK;
}

static int mlp_backward_dev(cudaStream_t st, const float* th, const float* X, const float* Y,
                            int n, MlpWork& w, float* g) {
  k_out_delta<<<nb((long long)n * H3), 256, 0, st>>>(w.y, Y, w.d3, n, H3);
  k_wgrad<<<nb(H3 * H2 + H3), 256, 0, st>>>(w.d3, w.a2, g + OFF_W3, g + OFF_B3, n, H2, H3);
  k_back_delta<<<nb((long long)n * H2), 256, 0, st>>>(th + OFF_W3, w.d3, w.a2, w.d2, n, H2, H3);
  k_wgrad<<<nb(H2 * H1 + H2), 256, 0, st>>>(w.d2, w.a1, g + OFF_W2, g + OFF_B2, n, H1, H2);
  k_back_delta<<<nb((long long)n * H1), 256, 0, st>>>(th + OFF_W2, w.d2, w.a1, w.d1, n, H1, H2);
  k_wgrad<<<nb(H1 * H0 + H1), 256, 0, st>>>(w.d1, X, g + OFF_W1, g + OFF_B1, n, H0, H1);
  g_kernels += 6;
  CK(cudaGetLastError());
  return DGFAS_OK;
}

static int work_alloc(MlpWork& w, int n) {
  float** ps[] = {&w.a1, &w.a2, &w.y, &w.d3, &w.d2, &w.d1};
  const int sz[] = {H1, H2, H3, H3, H2, H1};
  for (int q = 0; q < 6; ++q)
    if (cudaMalloc((void**)ps[q], (size_t)n * sz[q] * sizeof(float)) != cudaSuccess) {
      set_error("mlp work allocation");
      return DGFAS_ERR_OOM;
    }
  return DGFAS_OK;
}

static void work_free(MlpWork& w) {
  float* ps[] = {w.a1, w.a2, w.y, w.d3, w.d2, w.d1};
  for (float* p : ps)
    if (p) cudaFree(p);
}

extern "C" int dgfas_mlp_param_count(void) { return NPARAM; }

extern "C" int dgfas_mlp_forward(const float* params, const float* X, int n, float* out,
                                 void* stream) {
  if (!params || !X || !out || n <= 0) return DGFAS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  MlpWork w{};
  int rc = work_alloc(w, n);
  if (rc == DGFAS_OK) rc = mlp_forward_dev(st, params, X, n, w);
  if (rc == DGFAS_OK && cudaMemcpyAsync(out, w.y, (size_t)n * H3 * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    rc = DGFAS_ERR_CUDA;
  if (rc == DGFAS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = DGFAS_ERR_CUDA;
  work_free(w);
  return rc;
}

extern "C" int dgfas_mlp_grad(const float* params, const float* X, const float* Y, int n,
                              float* grad, void* stream) {
  if (!params || !X || !Y || !grad || n <= 0) return DGFAS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  MlpWork w{};
  int rc = work_alloc(w, n);
  if (rc == DGFAS_OK) rc = mlp_forward_dev(st, params, X, n, w);
  if (rc == DGFAS_OK) rc = mlp_backward_dev(st, params, X, Y, n, w, grad);
  if (rc == DGFAS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = DGFAS_ERR_CUDA;
  work_free(w);
  return rc;
}

// Minibatch Adam training.  X [n][24], Y [n][6] device FP32; params [NPARAM]
// device FP32, updated in place; m, v [NPARAM] device Adam moments (zero at
// the start of a run), t0 the number of steps already taken with them.
// Batches follow a host-side permutation per epoch (xorshift64 from `seed`).
// loss_out (host, may be NULL) receives the mean full-data loss after each epoch.
extern "C" int dgfas_mlp_train(float* params, float* m, float* v, const float* X, const float* Y,
                               int n, int epochs, int batch, float lr, unsigned long long seed,
                               int t0, float* loss_out, void* stream) {
  if (!params || !m || !v || !X || !Y || n <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0))
    return DGFAS_ERR_INVALID;
  if (batch > n) batch = n;
  cudaStream_t st = (cudaStream_t)stream;
  MlpWork w{}, wf{};
  float *xb = nullptr, *yb = nullptr, *g = nullptr;
  int* idx = nullptr;
  int rc = work_alloc(w, batch);
  if (rc == DGFAS_OK && loss_out) rc = work_alloc(wf, n);
  if (rc == DGFAS_OK && (cudaMalloc((void**)&xb, (size_t)batch * H0 * sizeof(float)) != cudaSuccess ||
                         cudaMalloc((void**)&yb, (size_t)batch * H3 * sizeof(float)) != cudaSuccess ||
                         cudaMalloc((void**)&g, NPARAM * sizeof(float)) != cudaSuccess ||
                         cudaMalloc((void**)&idx, (size_t)n * sizeof(int)) != cudaSuccess)) {
    set_error("mlp train allocation");
    rc = DGFAS_ERR_OOM;
  }
  std::vector<int> perm(n);
  unsigned long long s = seed ? seed : 88172645463325252ull;
  auto rnd = [&]() {
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    return s;
  };
  int t = t0;
  std::vector<float> yh;
  for (int ep = 0; ep < epochs && rc == DGFAS_OK; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[rnd() % (unsigned long long)(i + 1)]);
    if (cudaMemcpyAsync(idx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = DGFAS_ERR_CUDA;
      break;
    }
    for (int b0 = 0; b0 + batch <= n && rc == DGFAS_OK; b0 += batch) {
      k_gather_rows<<<nb((long long)batch * H0), 256, 0, st>>>(X, idx + b0, xb, batch, H0);
      k_gather_rows<<<nb((long long)batch * H3), 256, 0, st>>>(Y, idx + b0, yb, batch, H3);
      g_kernels += 2;
      rc = mlp_forward_dev(st, params, xb, batch, w);
      if (rc == DGFAS_OK) rc = mlp_backward_dev(st, params, xb, yb, batch, w, g);
      ++t;
      const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
      k_adam<<<nb(NPARAM), 256, 0, st>>>(params, g, m, v, NPARAM, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
      ++g_kernels;
    }
    if (rc == DGFAS_OK && loss_out) {
      rc = mlp_forward_dev(st, params, X, n, wf);
      if (rc == DGFAS_OK) {
        yh.resize((size_t)n * H3);
        std::vector<float> yt((size_t)n * H3);
        if (cudaMemcpyAsync(yh.data(), wf.y, yh.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(yt.data(), Y, yt.size() * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          rc = DGFAS_ERR_CUDA;
        } else {
          double acc = 0.0;
          for (size_t q = 0; q < yh.size(); ++q) acc += (double)(yh[q] - yt[q]) * (yh[q] - yt[q]);
          loss_out[ep] = (float)(acc / yh.size());
        }
      }
    }
  }
  if (rc == DGFAS_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = DGFAS_ERR_CUDA;
  work_free(w);
  work_free(wf);
  if (xb) cudaFree(xb);
  if (yb) cudaFree(yb);
  if (g) cudaFree(g);
  if (idx) cudaFree(idx);
  return rc;
}

// ---------------------------------------------------------------- inference on a level
// Per element: exact volume (2-point Gauss of det J), normalized corners.
__global__ void k_mlp_inputs(const double* __restrict__ corners, int ne, float* __restrict__ X,
                             double* __restrict__ vol) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double* cr = corners + (size_t)e * 24;
  const double gq = 0.57735026918962576451;   // 1/sqrt(3)
  double V = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {(q & 1) ? gq : -gq, (q & 2) ? gq : -gq, (q & 4) ? gq : -gq};
    double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < 8; ++c) {
      double s[3], f[3];
      for (int d = 0; d < 3; ++d) {
        s[d] = ((c >> d) & 1) ? 1.0 : -1.0;
        f[d] = 0.5 * (1.0 + s[d] * xi[d]);
      }
      const double dN[3] = {0.5 * s[0] * f[1] * f[2], 0.5 * s[1] * f[0] * f[2], 0.5 * s[2] * f[0] * f[1]};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) J[a * 3 + b] += dN[b] * cr[c * 3 + a];
    }
    V += J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
  }
  vol[e] = V;
  double cen[3] = {0, 0, 0};
  for (int c = 0; c < 8; ++c)
    for (int a = 0; a < 3; ++a) cen[a] += cr[c * 3 + a] / 8.0;
  const double sc = 1.0 / cbrt(V);
  for (int c = 0; c < 8; ++c)
    for (int a = 0; a < 3; ++a) X[(size_t)e * 24 + c * 3 + a] = (float)((cr[c * 3 + a] - cen[a]) * sc);
}

// The network's inputs of n elements: X [n][24] (device FP32) from corners
// [n][8][3] (device FP64); synchronizes `stream`.
extern "C" int dgfas_mlp_inputs(const double* corners, int n, float* X, void* stream) {
  if (!corners || !X || n <= 0) return DGFAS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  double* vol = nullptr;
  if (cudaMalloc((void**)&vol, (size_t)n * sizeof(double)) != cudaSuccess) {
    set_error("mlp inputs allocation");
    return DGFAS_ERR_OOM;
  }
  k_mlp_inputs<<<nb(n), 256, 0, st>>>(corners, n, X, vol);
  ++g_kernels;
  int rc = (cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess)
               ? DGFAS_OK : DGFAS_ERR_CUDA;
  cudaFree(vol);
  return rc;
}

// g_i = s_i nu dx_j dx_k / (2 dx_i) from the outputs; elements whose log
// scalings leave [-lmax, lmax] or are not finite keep the current (geometric)
// coefficients.  g[e][0] (the kappa term) is rescaled consistently.
__global__ void k_mlp_coeffs(const float* __restrict__ y, const double* __restrict__ vol,
                             int ne, double nu, double kappa, double lmax, double* __restrict__ g,
                             int* __restrict__ n_fallback) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const float* o = y + (size_t)e * 6;
  bool ok = true;
  for (int q = 0; q < 6; ++q) ok = ok && isfinite(o[q]);
  for (int q = 3; q < 6; ++q) ok = ok && fabs((double)o[q]) <= lmax;
  for (int q = 0; q < 3; ++q) ok = ok && fabs((double)o[q]) <= 5.0;
  if (!ok) {
    atomicAdd(n_fallback, 1);
    return;
  }
  const double h = cbrt(vol[e]);
  const double dx[3] = {exp((double)o[0]) * h, exp((double)o[1]) * h, exp((double)o[2]) * h};
  g[4 * e] = kappa * dx[0] * dx[1] * dx[2] / 8.0;
  for (int i = 0; i < 3; ++i)
    g[4 * e + 1 + i] = exp((double)o[3 + i]) * nu * dx[(i + 1) % 3] * dx[(i + 2) % 3] / (2.0 * dx[i]);
}

__global__ void k_g_to_float(const double* __restrict__ g, float* __restrict__ f, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) f[t] = (float)g[t];
}

// Replaces the surrogate coefficients of `level` by the MLP's prediction
// (params: trained weights, device FP32).  Returns the number of elements
// that fell back to the geometric surrogate in *n_fallback (host).
extern "C" int dgfas_learned_surrogate(void* ctx, int level, const float* params,
                                       double max_log_scaling, int* n_fallback) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !params || level < 0 || level >= (int)c->lv.size() || !(max_log_scaling > 0))
    return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  const int ne = H.ne;
  cudaStream_t st = c->stream;
  double *dcorn = nullptr, *vol = nullptr;
  float* X = nullptr;
  int* dfb = nullptr;
  MlpWork w{};
  int rc = work_alloc(w, ne);
  if (rc == DGFAS_OK && (cudaMalloc((void**)&dcorn, H.corners.size() * sizeof(double)) != cudaSuccess ||
                         cudaMalloc((void**)&vol, ne * sizeof(double)) != cudaSuccess ||
                         cudaMalloc((void**)&X, (size_t)ne * 24 * sizeof(float)) != cudaSuccess ||
                         cudaMalloc((void**)&dfb, sizeof(int)) != cudaSuccess)) {
    set_error("learned surrogate allocation");
    rc = DGFAS_ERR_OOM;
  }
  if (rc == DGFAS_OK) {
    cudaMemcpyAsync(dcorn, H.corners.data(), H.corners.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(dfb, 0, sizeof(int), st);
    k_mlp_inputs<<<nb(ne), 256, 0, st>>>(dcorn, ne, X, vol);
    ++g_kernels;
    rc = mlp_forward_dev(st, params, X, ne, w);
  }
  if (rc == DGFAS_OK) {
    k_mlp_coeffs<<<nb(ne), 256, 0, st>>>(w.y, vol, ne, c->nu, c->kappa, max_log_scaling, H.d_g, dfb);
    k_g_to_float<<<nb(4 * ne), 256, 0, st>>>(H.d_g, H.f_g, 4 * ne);
    g_kernels += 2;
    int hfb = 0;
    if (cudaMemcpyAsync(&hfb, dfb, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = DGFAS_ERR_CUDA;
    if (n_fallback) *n_fallback = hfb;
  }
  work_free(w);
  if (dcorn) cudaFree(dcorn);
  if (vol) cudaFree(vol);
  if (X) cudaFree(X);
  if (dfb) cudaFree(dfb);
  return rc;
}
