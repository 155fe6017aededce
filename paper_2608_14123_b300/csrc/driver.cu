// C ABI of the hot path: level setup, operator, smoother, FAS V-cycle (Alg. 2)
// and solve with crossover smoothing; CUDA-graph replay of the cycle body.
#include <algorithm>
#include <limits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "dgfas_internal.h"
#include "setup_host.h"

static thread_local std::string g_err;
void set_error(const std::string& s) { g_err = s; }

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #x); \
      return DGFAS_ERR_CUDA;                                                  \
    }                                                                         \
  } while (0)
#define RET(x)                    \
  do {                            \
    int rc_ = (x);                \
    if (rc_ != DGFAS_OK) return rc_; \
  } while (0)

template <typename T>
static int upload(T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return DGFAS_OK; }
  if (cudaMalloc((void**)dst, v.size() * sizeof(T)) != cudaSuccess) {
    set_error("cudaMalloc failed in setup");
    return DGFAS_ERR_OOM;
  }
  CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return DGFAS_OK;
}

template <typename T>
static int upload_f(float** dst, const std::vector<T>& v) {
  std::vector<float> f(v.begin(), v.end());
  return upload(dst, f);
}

static int dalloc(double** p, size_t n) {
  if (n == 0) { *p = nullptr; return DGFAS_OK; }
  if (cudaMalloc((void**)p, n * sizeof(double)) != cudaSuccess) {
    set_error("cudaMalloc failed");
    return DGFAS_ERR_OOM;
  }
  CK(cudaMemset(*p, 0, n * sizeof(double)));
  return DGFAS_OK;
}

// side type of a face: 0 interior, 1 Dirichlet, 2 Neumann, 3 interior face
// whose neighbour is frozen (the subdomain takes no layers from it)
static int side_idx(int nb, const std::vector<signed char>& cls) {
  if (nb >= 0) return cls[nb] == DGFAS_FROZEN ? 3 : 0;
  return nb == -1 ? 1 : 2;
}

// ---------------------------------------------------------------- one level
static int build_level(Ctx& c, const dgfas_level& in, const dgfas_params& prm, LevelHost& H) {
  const int p = in.p, N = p + 1, ne = in.n_elem;
  if (p < 1 || p > 10 || ne <= 0) {
    set_error("level: need 1 <= p <= 10 and n_elem > 0");
    return DGFAS_ERR_UNSUPPORTED;
  }
  H.p = p; H.N = N; H.ne = ne;
  H.ndof = (long long)ne * N * N * N;
  H.nbr.assign(in.nbr, in.nbr + 6 * (size_t)ne);
  H.nbr27.assign(in.nbr27, in.nbr27 + 27 * (size_t)ne);
  H.cls.assign(in.cls, in.cls + ne);
  H.corners.assign(in.corners, in.corners + 24 * (size_t)ne);
  H.parent.assign(in.parent, in.parent + ne);
  H.octant.assign(in.octant, in.octant + ne);
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f) {
      int nb = H.nbr[6 * e + f];
      if (nb >= ne || nb < -2) { set_error("nbr out of range"); return DGFAS_ERR_INVALID; }
    }
  for (size_t q = 0; q < H.nbr27.size(); ++q)
    if (H.nbr27[q] >= ne || H.nbr27[q] < -1) { set_error("nbr27 out of range"); return DGFAS_ERR_INVALID; }
  std::vector<double> x, w;
  host::gll(p, x, w);
  std::vector<double> D = host::diff_matrix(x);
  const int N2 = N * N, N3 = N2 * N;
  // box detection
  H.box = 1;
  std::vector<double> hbox(3 * (size_t)ne);
  for (int e = 0; e < ne && H.box; ++e) H.box = host::is_box(&H.corners[24 * e], &hbox[3 * e]);
  const double nu = c.nu;
  std::vector<double> G, fW, fc, mass, mu(6 * (size_t)ne), hp(6 * (size_t)ne);
  if (H.box) {
    for (int e = 0; e < ne; ++e)
      for (int f = 0; f < 6; ++f) hp[6 * e + f] = hbox[3 * e + f / 2];
  } else {
    G.assign((size_t)ne * 6 * N3, 0.0);
    fW.assign((size_t)ne * 6 * N2, 0.0);
    fc.assign((size_t)ne * 6 * 3 * N2, 0.0);
    mass.assign((size_t)ne * N3, 0.0);
    std::vector<double> Gi((size_t)N3 * 9), dJ(N3);
    for (int e = 0; e < ne; ++e) {
      const double* cr = &H.corners[24 * e];
      for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
          for (int i = 0; i < N; ++i) {
            const int n = (k * N + j) * N + i;
            double X[3], J[9];
            host::trilinear(cr, x[i], x[j], x[k], X, J);
            double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                         J[2] * (J[3] * J[7] - J[4] * J[6]);
            if (!(det > 0)) {
              set_error("non-positive Jacobian at a GLL node of element " + std::to_string(e));
              return DGFAS_ERR_MESH;
            }
            double* gi = &Gi[(size_t)n * 9];
            gi[0] = (J[4] * J[8] - J[5] * J[7]) / det;
            gi[1] = (J[2] * J[7] - J[1] * J[8]) / det;
            gi[2] = (J[1] * J[5] - J[2] * J[4]) / det;
            gi[3] = (J[5] * J[6] - J[3] * J[8]) / det;
            gi[4] = (J[0] * J[8] - J[2] * J[6]) / det;
            gi[5] = (J[2] * J[3] - J[0] * J[5]) / det;
            gi[6] = (J[3] * J[7] - J[4] * J[6]) / det;
            gi[7] = (J[1] * J[6] - J[0] * J[7]) / det;
            gi[8] = (J[0] * J[4] - J[1] * J[3]) / det;
            dJ[n] = det;
            const double wq = w[i] * w[j] * w[k];
            mass[(size_t)e * N3 + n] = wq * det;
            // G_df = nu w J grad xi_d . grad xi_f ; rows of gi are grad xi_b
            auto dot = [&](int d1, int d2) {
              return gi[3 * d1] * gi[3 * d2] + gi[3 * d1 + 1] * gi[3 * d2 + 1] + gi[3 * d1 + 2] * gi[3 * d2 + 2];
            };
            const double s = nu * wq * det;
            double* Ge = &G[(size_t)e * 6 * N3 + n];
            Ge[0] = s * dot(0, 0);
            Ge[N3] = s * dot(1, 1);
            Ge[2 * N3] = s * dot(2, 2);
            Ge[3 * N3] = s * dot(0, 1);
            Ge[4 * N3] = s * dot(0, 2);
            Ge[5 * N3] = s * dot(1, 2);
          }
      for (int f = 0; f < 6; ++f) {
        const int d = f / 2, side = f % 2, end = side ? N - 1 : 0;
        const double sg = side ? 1.0 : -1.0;
        // penalty length: the smallest local extent 2 / |grad xi_d| over the
        // face's GLL nodes (exactly h on a box)
        double hmin = 1e300;
        for (int b = 0; b < N; ++b)
          for (int a = 0; a < N; ++a) {
            int i, j, k;
            if (d == 0) { i = end; j = a; k = b; }
            else if (d == 1) { i = a; j = end; k = b; }
            else { i = a; j = b; k = end; }
            const int n = (k * N + j) * N + i;
            const double* gi = &Gi[(size_t)n * 9];
            const double gd2 = gi[3 * d] * gi[3 * d] + gi[3 * d + 1] * gi[3 * d + 1] + gi[3 * d + 2] * gi[3 * d + 2];
            const double wab = w[a] * w[b];
            const double Wq = wab * dJ[n] * std::sqrt(gd2);
            fW[((size_t)e * 6 + f) * N2 + b * N + a] = Wq;
            hmin = std::min(hmin, 2.0 / std::sqrt(gd2));
            for (int t = 0; t < 3; ++t) {
              const double gdt = gi[3 * d] * gi[3 * t] + gi[3 * d + 1] * gi[3 * t + 1] + gi[3 * d + 2] * gi[3 * t + 2];
              fc[(((size_t)e * 6 + f) * 3 + t) * N2 + b * N + a] = sg * nu * wab * dJ[n] * gdt;
            }
          }
        hp[6 * e + f] = hmin;
      }
    }
  }
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f) {
      const int nb = H.nbr[6 * e + f];
      const double own = p * (p + 1) / (2.0 * hp[6 * e + f]);
      if (nb >= 0) {
        const double oth = p * (p + 1) / (2.0 * hp[6 * nb + (f ^ 1)]);
        mu[6 * e + f] = prm.mu_star * 0.5 * (own + oth);
      } else {
        mu[6 * e + f] = prm.mu_star * own;
      }
    }
  // ---- Schwarz tables
  H.m = host::overlap_layers(p, prm.delta);
  if (H.m < 1 || H.m >= N) { set_error("overlap layers must satisfy 1 <= m < p+1"); return DGFAS_ERR_UNSUPPORTED; }
  H.nsm = N + 2 * H.m;
  if (H.nsm > DGFAS_MAX_NS) { set_error("subdomain width > 16"); return DGFAS_ERR_UNSUPPORTED; }
  const int nsm = H.nsm;
  std::vector<double> S(16 * (size_t)nsm * nsm, 0.0), lam(16 * (size_t)nsm, 0.0),
      Wt(16 * (size_t)nsm, 0.0);
  const char sc[4] = {'i', 'd', 'n', 'f'};
  for (int v = 0; v < 16; ++v) {
    std::vector<double> Sv, lv, wv;
    host::fd_variant(p, H.m, prm.mu_star, prm.delta, sc[v / 4], sc[v % 4], Sv, lv, wv);
    const int n = (int)lv.size();
    for (int r = 0; r < n; ++r) {
      for (int q = 0; q < n; ++q) S[((size_t)v * nsm + r) * nsm + q] = Sv[r * n + q];
      lam[v * nsm + r] = lv[r];
      Wt[v * nsm + r] = wv[r];
    }
    for (int r = n; r < nsm; ++r) lam[v * nsm + r] = 1.0;   // padding, never read as divisor
  }
  std::vector<unsigned char> var(3 * (size_t)ne);
  std::vector<double> g(4 * (size_t)ne);
  for (int e = 0; e < ne; ++e) {
    for (int d = 0; d < 3; ++d)
      var[3 * e + d] = (unsigned char)(4 * side_idx(H.nbr[6 * e + 2 * d], H.cls) +
                                       side_idx(H.nbr[6 * e + 2 * d + 1], H.cls));
    double dx[3];
    host::surrogate_widths(&H.corners[24 * e], dx);
    g[4 * e] = c.kappa * dx[0] * dx[1] * dx[2] / 8.0;
    for (int i = 0; i < 3; ++i) g[4 * e + 1 + i] = nu * dx[(i + 1) % 3] * dx[(i + 2) % 3] / (2.0 * dx[i]);
  }
  // combine offsets: for element e and neighbour slot (ox, oy, oz) the patch
  // index of e's node (0, 0, 0) inside that neighbour's weighted patch (the
  // neighbour's index NS^3 plus the shift of e's nodes in its subdomain), or
  // the sentinel (the type's minimum) when the slot contributes nothing: no
  // neighbour, a frozen one, or a side of the neighbour without layers
  {
    const long long NS3 = (long long)nsm * nsm * nsm;
    std::vector<long long> off(27 * (size_t)ne, std::numeric_limits<long long>::min());
    for (int e = 0; e < ne; ++e)
      for (int slot = 0; slot < 27; ++slot) {
        const int src = H.nbr27[27 * (size_t)e + slot];
        if (src < 0 || H.cls[src] == DGFAS_FROZEN) continue;
        const int o[3] = {slot % 3 - 1, (slot / 3) % 3 - 1, slot / 9 - 1};
        int shift[3];
        bool reach = true;
        for (int d = 0; d < 3; ++d) {
          const int v = var[3 * (size_t)src + d];
          const bool left_i = (v >> 2) == 0, right_i = (v & 3) == 0;
          const int ml = left_i ? H.m : 0;   // the neighbour's left layers
          if ((o[d] < 0 && !right_i) || (o[d] > 0 && !left_i)) reach = false;
          shift[d] = o[d] == 0 ? ml : (o[d] < 0 ? ml + N : -(N - H.m));
        }
        if (reach)
          off[27 * (size_t)e + slot] =
              (long long)src * NS3 + ((long long)shift[2] * nsm + shift[1]) * nsm + shift[0];
      }
    H.coff32 = (long long)ne * NS3 < (1LL << 31);
    if (H.coff32) {
      std::vector<int> o32(off.size());
      for (size_t t = 0; t < off.size(); ++t)
        o32[t] = off[t] == std::numeric_limits<long long>::min() ? std::numeric_limits<int>::min()
                                                                  : (int)off[t];
      RET(upload(&H.d_coff32, o32));
    } else {
      RET(upload(&H.d_coff64, off));
    }
  }
  // ---- uploads
  RET(upload(&H.d_nbr, H.nbr));
  RET(upload(&H.d_nbr27, H.nbr27));
  RET(upload(&H.d_cls, H.cls));
  RET(upload(&H.d_var, var));
  RET(upload(&H.d_D, D));
  RET(upload(&H.d_w, w));
  RET(upload(&H.d_x, x));
  RET(upload(&H.d_mu, mu));
  RET(upload(&H.d_g, g));
  RET(upload(&H.d_S, S));
  RET(upload(&H.d_lam, lam));
  RET(upload(&H.d_W, Wt));
  RET(upload_f(&H.f_D, D));
  RET(upload_f(&H.f_w, w));
  RET(upload_f(&H.f_x, x));
  RET(upload_f(&H.f_mu, mu));
  RET(upload_f(&H.f_g, g));
  RET(upload_f(&H.f_S, S));
  RET(upload_f(&H.f_lam, lam));
  RET(upload_f(&H.f_W, Wt));
  {
    std::vector<double> Lh((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        for (int q = 0; q < N; ++q) Lh[i * N + j] += D[q * N + i] * w[q] * D[q * N + j];
    RET(upload(&H.d_Lhat, Lh));
    RET(upload_f(&H.f_Lhat, Lh));
  }
  if (H.box) {
    RET(upload(&H.d_h, hbox));
    RET(upload_f(&H.f_h, hbox));
    std::vector<double> bx(6 * (size_t)ne);
    for (int e = 0; e < ne; ++e)
      for (int dd = 0; dd < 3; ++dd) {
        const double hj = hbox[3 * e + (dd + 1) % 3], hk = hbox[3 * e + (dd + 2) % 3];
        bx[6 * e + dd] = nu * hj * hk / (2.0 * hbox[3 * e + dd]);
        bx[6 * e + 3 + dd] = nu * hj * hk / 4.0;
      }
    RET(upload(&H.d_bx, bx));
    RET(upload_f(&H.f_bx, bx));
  } else {
    // coefficients of the trilinear map in monomial form (the FP32 operator
    // recomputes the metric from them instead of reading it)
    std::vector<double> tri(24 * (size_t)ne, 0.0);
    for (int e = 0; e < ne; ++e)
      for (int c = 0; c < 8; ++c) {
        const double s0 = (c & 1) ? 1.0 : -1.0, s1 = (c & 2) ? 1.0 : -1.0,
                     s2 = (c & 4) ? 1.0 : -1.0;
        const double sg[7] = {s0, s1, s2, s0 * s1, s0 * s2, s1 * s2, s0 * s1 * s2};
        for (int k = 0; k < 7; ++k)
          for (int a = 0; a < 3; ++a)
            tri[24 * (size_t)e + 3 * k + a] += 0.125 * sg[k] * H.corners[24 * (size_t)e + 3 * c + a];
      }
    RET(upload(&H.d_tri, tri));
    RET(upload_f(&H.f_tri, tri));
    RET(upload(&H.d_G, G));
    RET(upload(&H.d_fW, fW));
    RET(upload(&H.d_fc, fc));
    RET(upload(&H.d_mass, mass));
    RET(upload_f(&H.f_G, G));
    RET(upload_f(&H.f_fW, fW));
    RET(upload_f(&H.f_fc, fc));
    RET(upload_f(&H.f_mass, mass));
  }
  auto fill = [&](auto& V, auto* bx_, auto* Lh_, auto* h, auto* G_, auto* fW_, auto* fc_, auto* mu_, auto* mass_, auto* D_,
                  auto* w_, auto* x_, auto* g_, auto* S_, auto* lam_, auto* W_) {
    V.ne = ne; V.N = N; V.m = H.m; V.nsm = nsm; V.box = H.box;
    V.nu = nu; V.kappa = c.kappa;
    V.nbr = H.d_nbr; V.nbr27 = H.d_nbr27; V.cls = H.d_cls; V.var = H.d_var;
    V.bx = bx_; V.Lhat = Lh_; V.h = h; V.G = G_; V.fW = fW_; V.fc = fc_; V.mu = mu_; V.mass = mass_; V.D = D_; V.w = w_;
    V.x = x_; V.g = g_; V.S = S_; V.lam = lam_; V.W = W_;
    V.Btc = H.d_Btc;
  };
  {
    // tensor-core FD operand tiles, one pair per variant: tile 0 holds S^T
    // (entry (n, k) = S[k][n]), tile 1 holds S (entry (n, k) = S[n][k]), both
    // zero padded to 16 x 16 BF16 in the K-major no-swizzle layout (byte
    // (n/8) 256 + (k/8) 128 + (n%8) 16 + (k%8) 2)
    std::vector<__nv_bfloat16> tiles(16 * 2 * 256, __float2bfloat16(0.0f));
    for (int v = 0; v < 16; ++v) {
      const int nv = H.N + H.m * (((v >> 2) == 0) + ((v & 3) == 0));
      for (int n = 0; n < nv; ++n)
        for (int k = 0; k < nv; ++k) {
          const size_t o = (size_t)((n >> 3) * 128 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7));
          const float st = (float)S[((size_t)v * nsm + k) * nsm + n];
          const float sn = (float)S[((size_t)v * nsm + n) * nsm + k];
          tiles[(size_t)(2 * v) * 256 + o] = __float2bfloat16(st);
          tiles[(size_t)(2 * v + 1) * 256 + o] = __float2bfloat16(sn);
        }
    }
    if (cudaMalloc((void**)&H.d_Btc, tiles.size() * sizeof(__nv_bfloat16)) != cudaSuccess) {
      set_error("cudaMalloc failed in setup");
      return DGFAS_ERR_OOM;
    }
    CK(cudaMemcpy(H.d_Btc, tiles.data(), tiles.size() * sizeof(__nv_bfloat16),
                  cudaMemcpyHostToDevice));
  }
  fill(H.v64, H.d_bx, H.d_Lhat, H.d_h, H.d_G, H.d_fW, H.d_fc, H.d_mu, H.d_mass, H.d_D, H.d_w, H.d_x, H.d_g, H.d_S,
       H.d_lam, H.d_W);
  fill(H.v32, H.f_bx, H.f_Lhat, H.f_h, H.f_G, H.f_fW, H.f_fc, H.f_mu, H.f_mass, H.f_D, H.f_w, H.f_x, H.f_g, H.f_S,
       H.f_lam, H.f_W);
  H.v64.tri = H.d_tri;
  H.v32.tri = H.f_tri;
  H.v64.coff = H.v32.coff = H.coff32 ? (const void*)H.d_coff32 : (const void*)H.d_coff64;
  return DGFAS_OK;
}

// transfer matrices from level C (coarse) to level F (fine)
// x = A^-1 B for a small dense SPD A [n][n] and B [n][m] (row-major), by
// Gauss-Jordan elimination without pivoting (the matrices here are Gram
// matrices of interpolation operators, well conditioned for n <= 11)
static std::vector<double> small_solve(std::vector<double> A, std::vector<double> B, int n, int m) {
  for (int k = 0; k < n; ++k) {
    const double piv = A[k * n + k];
    for (int j = 0; j < n; ++j) A[k * n + j] /= piv;
    for (int j = 0; j < m; ++j) B[k * m + j] /= piv;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A[i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < m; ++j) B[i * m + j] -= f * B[k * m + j];
    }
  }
  return B;
}

// L2 projection matrices of P (reference coordinates, fine GLL quadrature):
// I [ns][Nf][Nc] the interpolation of each child side (ns = 2 for h, 1 for
// p), w the fine GLL weights; P_s = M^-1 c I_s^T W with M = c sum_s I_s^T W
// I_s and c = 1/ns (each h-child covers half of the parent's width).
static void l2_projection(const std::vector<double>& I, const std::vector<double>& w, int ns,
                          int Nf, int Nc, std::vector<double>& P) {
  const double cw = 1.0 / ns;
  std::vector<double> M((size_t)Nc * Nc, 0.0);
  for (int s = 0; s < ns; ++s)
    for (int a = 0; a < Nc; ++a)
      for (int b = 0; b < Nc; ++b)
        for (int i = 0; i < Nf; ++i)
          M[a * Nc + b] += cw * I[((size_t)s * Nf + i) * Nc + a] * w[i] * I[((size_t)s * Nf + i) * Nc + b];
  for (int s = 0; s < ns; ++s) {
    std::vector<double> B((size_t)Nc * Nf);
    for (int a = 0; a < Nc; ++a)
      for (int i = 0; i < Nf; ++i) B[a * Nf + i] = cw * I[((size_t)s * Nf + i) * Nc + a] * w[i];
    std::vector<double> X = small_solve(M, B, Nc, Nf);
    std::copy(X.begin(), X.end(), P.begin() + (size_t)s * Nc * Nf);
  }
}

static int build_transfer(LevelHost& C, LevelHost& F, int projection) {
  const int Nf = F.N, Nc = C.N;
  bool h = true, pref = true;
  for (int e = 0; e < F.ne; ++e) {
    if (F.octant[e] < 0) h = false; else pref = false;
    if (F.parent[e] < 0 || F.parent[e] >= C.ne) { set_error("parent out of range"); return DGFAS_ERR_INVALID; }
  }
  if (!h && !pref) { set_error("a level mixes h- and p-children"); return DGFAS_ERR_INVALID; }
  if (h && Nf != Nc) { set_error("h-refinement must keep the degree"); return DGFAS_ERR_INVALID; }
  std::vector<double> xf, wf, xc, wc;
  host::gll(F.p, xf, wf);
  host::gll(C.p, xc, wc);
  std::vector<double> I(2 * (size_t)Nf * Nc, 0.0), P(2 * (size_t)Nc * Nf, 0.0);
  for (int s = 0; s < 2; ++s) {
    std::vector<double> y(Nf);
    for (int i = 0; i < Nf; ++i) y[i] = h ? 0.5 * (xf[i] + (s ? 1.0 : -1.0)) : xf[i];
    std::vector<double> Ls = host::interp(xc, y);   // [Nf][Nc]
    std::copy(Ls.begin(), Ls.end(), I.begin() + (size_t)s * Nf * Nc);
    std::vector<double> yc(Nc), wgt(Nc);
    for (int i = 0; i < Nc; ++i) {
      if (!h) { yc[i] = xc[i]; wgt[i] = 1.0; continue; }
      const bool inside = s ? xc[i] >= 0.0 : xc[i] <= 0.0;
      wgt[i] = inside ? (xc[i] == 0.0 ? 0.5 : 1.0) : 0.0;
      double t = 2.0 * xc[i] - (s ? 1.0 : -1.0);
      yc[i] = std::min(1.0, std::max(-1.0, t));
    }
    std::vector<double> Lp = host::interp(xf, yc);  // [Nc][Nf]
    for (int i = 0; i < Nc; ++i)
      for (int j = 0; j < Nf; ++j) P[((size_t)s * Nc + i) * Nf + j] = wgt[i] * Lp[i * Nf + j];
  }
  if (projection == DGFAS_P_L2) l2_projection(I, wf, h ? 2 : 1, Nf, Nc, P);
  std::vector<int> children(8 * (size_t)C.ne, -1);
  for (int e = 0; e < F.ne; ++e) {
    int slot = h ? F.octant[e] : 0;
    if (slot < 0 || slot > 7) { set_error("octant out of range"); return DGFAS_ERR_INVALID; }
    children[8 * (size_t)F.parent[e] + slot] = e;
  }
  RET(upload(&F.d_I, I));
  RET(upload(&F.d_P, P));
  RET(upload(&F.d_children, children));
  RET(upload(&F.d_parent, F.parent));
  RET(upload(&F.d_octant, F.octant));
  F.tr.nef = F.ne; F.tr.nec = C.ne; F.tr.Nf = Nf; F.tr.Nc = Nc; F.tr.h = h ? 1 : 0;
  // a p-transfer between symmetric GLL node sets has centrosymmetric matrices
  // (M[n-1-r][m-1-c] = M[r][c]); the even-odd transfer kernels rely on it
  F.tr.cs = 0;
  if (!h) {
    double dev = 0.0, big = 0.0;
    for (int r = 0; r < Nf; ++r)
      for (int q = 0; q < Nc; ++q) {
        dev = std::max(dev, std::fabs(I[r * Nc + q] - I[(Nf - 1 - r) * Nc + (Nc - 1 - q)]));
        big = std::max(big, std::fabs(I[r * Nc + q]));
      }
    for (int r = 0; r < Nc; ++r)
      for (int q = 0; q < Nf; ++q) {
        dev = std::max(dev, std::fabs(P[r * Nf + q] - P[(Nc - 1 - r) * Nf + (Nf - 1 - q)]));
        big = std::max(big, std::fabs(P[r * Nf + q]));
      }
    F.tr.cs = dev <= 1e-13 * big ? 1 : 0;
  }
  RET(prepare_transfer(F.tr));
  F.tr.parent = F.d_parent; F.tr.octant = F.d_octant; F.tr.children = F.d_children;
  F.tr.clsf = F.d_cls; F.tr.I = F.d_I; F.tr.P = F.d_P;
  return DGFAS_OK;
}

// explicit inverse of the (SPD) root operator: columns A e_i by the apply
// kernel, then symmetrization and in-place Gauss-Jordan inversion on the GPU
// (no pivoting: the pivots of an SPD matrix stay positive; a non-positive one
// is reported)
static int build_root(Ctx& c) {
  LevelHost& R = c.lv[0];
  const int n = (int)R.ndof;
  if (n > DGFAS_MAX_ROOT) {
    set_error("root level larger than " + std::to_string(DGFAS_MAX_ROOT) + " DoF");
    return DGFAS_ERR_UNSUPPORTED;
  }
  c.n_root = n;
  double *E = nullptr, *A = nullptr, *work = nullptr;
  int* flag = nullptr;
  RET(dalloc(&E, (size_t)n * n));
  RET(dalloc(&A, (size_t)n * n));
  RET(dalloc(&work, 2 * (size_t)n));
  if (cudaMalloc((void**)&flag, sizeof(int)) != cudaSuccess) {
    set_error("cudaMalloc failed in setup");
    return DGFAS_ERR_OOM;
  }
  RET(launch_identity(c, E, n));
  for (int i = 0; i < n; ++i)
    RET(launch_apply(c, 0, DGFAS_FP64, E + (size_t)i * n, nullptr, A + (size_t)i * n, 1.0));
  // kappa = 0 without Dirichlet faces (periodic or pure Neumann): the constants
  // span the null space; invert A + c 1 1^T, which for a consistent right-hand
  // side (1^T g = 0) returns the solution with 1^T u = 0
  bool dirichlet = false;
  for (int v : R.nbr) dirichlet |= v == -1;
  double shift = 0.0;
  if (c.kappa == 0.0 && !dirichlet) {
    std::vector<double> diag(n);
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaMemcpy2D(diag.data(), sizeof(double), A, (size_t)(n + 1) * sizeof(double),
                    sizeof(double), n, cudaMemcpyDeviceToHost));
    double tr = 0.0;
    for (double v : diag) tr += v;
    shift = tr / n / n;
  }
  int rc = launch_root_inverse(c, A, n, shift, work, flag);
  int bad = 0;
  if (rc == DGFAS_OK) {
    CK(cudaStreamSynchronize(c.stream));
    CK(cudaMemcpy(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost));
  }
  cudaFree(E);
  cudaFree(work);
  cudaFree(flag);
  if (rc != DGFAS_OK) { cudaFree(A); return rc; }
  if (bad) {
    cudaFree(A);
    set_error("root operator not positive definite");
    return DGFAS_ERR_MESH;
  }
  c.Ainv = A;
  return DGFAS_OK;
}

static void free_level(LevelHost& H) {
  void* ptrs[] = {H.d_Btc, H.d_bx, H.d_Lhat, H.f_bx, H.f_Lhat, H.d_nbr, H.d_nbr27, H.d_parent, H.d_octant, H.d_children, H.d_cls, H.d_var,
                  H.d_h, H.d_G, H.d_fW, H.d_fc, H.d_mu, H.d_mass, H.d_D, H.d_w, H.d_g, H.d_S,
                  H.d_lam, H.d_W, H.d_x, H.f_h, H.f_G, H.f_fW, H.f_fc, H.f_mu, H.f_mass, H.f_D,
                  H.f_w, H.f_g, H.f_S, H.f_lam, H.f_W, H.f_x, H.d_I, H.d_P, H.u, H.gv, H.r,
                  H.ubar, H.t, H.delta, H.fl, H.d_tri, H.f_tri, H.d_coff32, H.d_coff64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

extern "C" void dgfas_destroy(void* vctx) {
  if (!vctx) return;
  Ctx* c = (Ctx*)vctx;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(*c);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  for (auto& H : c->lv) free_level(H);
  void* ptrs[] = {c->patch, c->rw, c->red, c->scg_buf, c->dscal, c->dcnt, c->Ainv, c->tc_err,
                  c->apply_scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->red_host) cudaFreeHost(c->red_host);
  delete c;
}

// Host-only checks of one level's input arrays (no device work).  The
// kernels read a neighbour's data through its opposite face (f ^ 1) in the
// same face-local node order, so the face-neighbour relation must be
// reciprocal through the opposite face and the two elements' face corners
// must coincide corner by corner, up to one translation (periodic meshes
// identify opposite boundary faces by a translation): aligned local axes.
static int check_level(const dgfas_level& in, int l) {
  if (!in.corners || !in.nbr || !in.nbr27 || !in.cls || (l > 0 && (!in.parent || !in.octant))) {
    set_error("setup: level arrays missing");
    return DGFAS_ERR_INVALID;
  }
  if (in.p < 1 || in.p > 10 || in.n_elem <= 0) {
    set_error("level: need 1 <= p <= 10 and n_elem > 0");
    return DGFAS_ERR_UNSUPPORTED;
  }
  const int ne = in.n_elem;
  for (size_t q = 0; q < 27 * (size_t)ne; ++q)
    if (in.nbr27[q] >= ne || in.nbr27[q] < -1) {
      set_error("nbr27 out of range");
      return DGFAS_ERR_INVALID;
    }
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 6; ++f) {
      const int nb = in.nbr[6 * e + f];
      if (nb >= ne || nb < -2) {
        set_error("nbr out of range");
        return DGFAS_ERR_INVALID;
      }
    }
  // the 27-neighbourhood (read by the Schwarz gather and combine) must agree
  // with the face neighbours: the centre slot is the element itself, a face
  // slot holds the face neighbour or -1 on a boundary face
  for (int e = 0; e < ne; ++e) {
    const int* n27 = in.nbr27 + 27 * (size_t)e;
    if (n27[13] != e) {
      set_error("level " + std::to_string(l) + ": nbr27 centre slot of element " +
                std::to_string(e) + " is not the element");
      return DGFAS_ERR_INVALID;
    }
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, o = (f & 1) ? 2 : 0;
      const int slot = d == 0 ? o + 3 + 9 : (d == 1 ? 1 + 3 * o + 9 : 1 + 3 + 9 * o);
      const int nb = in.nbr[6 * e + f];
      if (n27[slot] != (nb >= 0 ? nb : -1)) {
        set_error("level " + std::to_string(l) + ": nbr27 face slot " + std::to_string(slot) +
                  " of element " + std::to_string(e) + " disagrees with face neighbour " +
                  std::to_string(nb));
        return DGFAS_ERR_INVALID;
      }
    }
  }
  for (int e = 0; e < ne; ++e) {
    const double* xe = in.corners + 24 * (size_t)e;
    double scale = 0.0;   // the element's largest corner-to-corner extent
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < 3; ++k) scale = std::max(scale, std::fabs(xe[3 * c + k] - xe[k]));
    for (int f = 0; f < 6; ++f) {
      const int nb = in.nbr[6 * e + f];
      if (nb < 0) continue;
      if (in.nbr[6 * (size_t)nb + (f ^ 1)] != e) {
        set_error("level " + std::to_string(l) + ": face " + std::to_string(f) + " of element " +
                  std::to_string(e) + " has neighbour " + std::to_string(nb) +
                  ", whose opposite face does not point back");
        return DGFAS_ERR_MESH;
      }
      const int d = f >> 1, side = f & 1;
      const double* xn = in.corners + 24 * (size_t)nb;
      double t0[3] = {0, 0, 0};
      bool first = true;
      for (int c = 0; c < 8; ++c) {
        if (((c >> d) & 1) != side) continue;
        const int cn = c ^ (1 << d);
        double t[3];
        for (int k = 0; k < 3; ++k) t[k] = xe[3 * c + k] - xn[3 * cn + k];
        if (first) {
          for (int k = 0; k < 3; ++k) t0[k] = t[k];
          first = false;
        } else {
          for (int k = 0; k < 3; ++k)
            if (std::fabs(t[k] - t0[k]) > 1e-8 * scale) {
              set_error("level " + std::to_string(l) + ": face " + std::to_string(f) +
                        " of element " + std::to_string(e) + " and the opposite face of element " +
                        std::to_string(nb) +
                        " do not coincide corner by corner (neighbours must share aligned local axes)");
              return DGFAS_ERR_MESH;
            }
        }
      }
    }
  }
  return DGFAS_OK;
}

extern "C" int dgfas_check_mesh(const dgfas_mesh* mesh) {
  if (!mesh || mesh->n_levels < 1 || !mesh->levels) {
    set_error("check_mesh: null argument or no levels");
    return DGFAS_ERR_INVALID;
  }
  for (int l = 0; l < mesh->n_levels; ++l) {
    const int rc = check_level(mesh->levels[l], l);
    if (rc != DGFAS_OK) return rc;
  }
  return DGFAS_OK;
}

extern "C" int dgfas_setup_levels(const dgfas_mesh* mesh, const dgfas_params* prm,
                                  void* stream, void** out) {
  if (!mesh || !prm || !out || mesh->n_levels < 1 || !mesh->levels) {
    set_error("setup: null argument or no levels");
    return DGFAS_ERR_INVALID;
  }
  if (!(prm->delta > 0 && prm->delta < 0.5) || !(prm->mu_star > 0) || prm->s1 < 0 ||
      prm->s2 < 0 || prm->sc < 0 || !(mesh->nu > 0) || mesh->kappa < 0) {
    set_error("setup: parameter out of range");
    return DGFAS_ERR_INVALID;
  }
  if (prm->precision != DGFAS_FP64 && prm->precision != DGFAS_FP32 &&
      prm->precision != DGFAS_BF16) {
    set_error("setup: unknown precision");
    return DGFAS_ERR_INVALID;
  }
  if (prm->coarse != DGFAS_COARSE_DENSE && prm->coarse != DGFAS_COARSE_SCG) {
    set_error("setup: unknown root solver");
    return DGFAS_ERR_INVALID;
  }
  if (prm->projection != DGFAS_P_INTERP && prm->projection != DGFAS_P_L2) {
    set_error("setup: unknown solution projection");
    return DGFAS_ERR_INVALID;
  }
  {
    const int rc = dgfas_check_mesh(mesh);   // host-only, before any device work
    if (rc != DGFAS_OK) return rc;
  }
  Ctx* c = new Ctx();
  c->stream = (cudaStream_t)stream;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
      set_error("setup: no CUDA device");
      delete c;
      return DGFAS_ERR_CUDA;
    }
    c->red_blocks = 4 * sms;
  }
  c->prm = *prm;
  if (!(c->prm.root_rtol > 0)) c->prm.root_rtol = 1e-3;
  if (c->prm.root_steps <= 0) c->prm.root_steps = 64;
  c->nu = mesh->nu;
  c->kappa = mesh->kappa;
  c->lv.resize(mesh->n_levels);
  int rc = DGFAS_OK;
  size_t patch = 0, maxdof = 0;
  for (int l = 0; l < mesh->n_levels && rc == DGFAS_OK; ++l) {
    const dgfas_level& in = mesh->levels[l];
    if (!in.corners || !in.nbr || !in.nbr27 || !in.cls || (l > 0 && (!in.parent || !in.octant))) {
      set_error("setup: level arrays missing");
      rc = DGFAS_ERR_INVALID;
      break;
    }
    rc = build_level(*c, in, *prm, c->lv[l]);
    if (rc != DGFAS_OK) break;
    LevelHost& H = c->lv[l];
    patch = std::max(patch, (size_t)H.ne * H.nsm * H.nsm * H.nsm * sizeof(double));
    maxdof = std::max(maxdof, (size_t)H.ndof);
    if (l > 0) rc = build_transfer(c->lv[l - 1], H, prm->projection);
    if (rc != DGFAS_OK) break;
    const bool top = l == mesh->n_levels - 1;
    if (!top) {
      rc = dalloc(&H.u, H.ndof);
      if (!rc) rc = dalloc(&H.gv, H.ndof);
      if (!rc) rc = dalloc(&H.ubar, H.ndof);
      if (!rc) rc = dalloc(&H.t, H.ndof);
    }
    if (!rc) rc = dalloc(&H.r, H.ndof);
    if (!rc) rc = dalloc(&H.delta, H.ndof);
    for (int e = 0; e < H.ne; ++e) {
      H.has_leaf |= H.cls[e] == DGFAS_LEAF;
      H.has_frozen |= H.cls[e] == DGFAS_FROZEN;
    }
    if (!rc && !top && H.has_leaf) rc = dalloc(&H.fl, H.ndof);
    if ((!top && H.has_leaf) || H.has_frozen) c->local = 1;
  }
  if (rc == DGFAS_OK) {
    if (cudaMalloc(&c->patch, patch) != cudaSuccess) { set_error("patch buffer"); rc = DGFAS_ERR_OOM; }
    c->patch_bytes = patch;
  }
  if (rc == DGFAS_OK && cudaMalloc(&c->rw, maxdof * sizeof(double)) != cudaSuccess) {
    set_error("smoother residual buffer");
    rc = DGFAS_ERR_OOM;
  }
  if (rc == DGFAS_OK && (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess)) {
    set_error("stream/event creation");
    rc = DGFAS_ERR_CUDA;
  }
  if (rc == DGFAS_OK) rc = dalloc(&c->red, 5 * c->red_blocks + 64);
  if (rc == DGFAS_OK && cudaMallocHost((void**)&c->red_host, (5 * c->red_blocks + 64) * sizeof(double)) != cudaSuccess) {
    set_error("pinned host buffer");
    rc = DGFAS_ERR_OOM;
  }
  if (rc == DGFAS_OK && (prm->smoother == DGFAS_SCG || prm->coarse == DGFAS_COARSE_SCG))
    rc = dalloc(&c->scg_buf, 4 * (maxdof + kScgPad) + 64);
  if (rc == DGFAS_OK) {
    size_t need = 0;
    for (const LevelHost& H : c->lv)
      if (!H.box) need = std::max(need, (size_t)H.ne * (3 * H.N * H.N * H.N + 12 * H.N * H.N));
    if (need > 0) {
      rc = dalloc(&c->apply_scratch, need);
      c->apply_scratch_n = need;
    }
  }
  if (rc == DGFAS_OK) rc = dalloc(&c->dscal, 64);
  if (rc == DGFAS_OK) {
    if (cudaMalloc((void**)&c->dcnt, 8 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->dcnt, 0, 8 * sizeof(int)) != cudaSuccess) {
      set_error("reduction counters");
      rc = DGFAS_ERR_OOM;
    }
  }
  if (rc == DGFAS_OK) {
    if (cudaMalloc((void**)&c->tc_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->tc_err, 0, sizeof(int)) != cudaSuccess) {
      set_error("error flag");
      rc = DGFAS_ERR_OOM;
    }
  }
  if (rc == DGFAS_OK && prm->coarse != DGFAS_COARSE_SCG) rc = build_root(*c);
  if (rc != DGFAS_OK) {
    dgfas_destroy(c);
    return rc;
  }
  *out = c;
  return DGFAS_OK;
}

// ---------------------------------------------------------------- reductions
static int norm_dev(Ctx& c, const double* v, long long n, double* out) {
  RET(launch_sumsq(c, v, n, c.red));
  CK(cudaMemcpyAsync(c.red_host, c.red, c.red_blocks * sizeof(double), cudaMemcpyDeviceToHost,
                     c.stream));
  CK(cudaStreamSynchronize(c.stream));
  double s = 0.0;
  for (int i = 0; i < c.red_blocks; ++i) s += c.red_host[i];
  *out = std::sqrt(s);
  return DGFAS_OK;
}

// ---------------------------------------------------------------- smoothers
// Schwarz correction of the smoother-precision residual in c.rw: delta += z.
static int schwarz_into_delta(Ctx& c, int l) {
  const int prec = c.prm.precision;
  RET(launch_fd(c, l, prec, c.rw));
  return launch_combine(c, l, prec, c.lv[l].delta);
}

// One smoothing block of n WAS sweeps (Alg. 5) in correction form.  lv[l].r
// holds the FP64 residual r = g - A u of the current u; the sweeps solve
// A delta = r approximately in the smoother precision, starting from delta = 0
// (zero_start) or from the prolongated correction already in lv[l].delta, and
// finally u += delta.  Each sweep: w = r - A delta, delta += sum_e R^T W A~^-1 R w.
// With want_res, lv[l].r becomes the residual r - A delta of the new u.  In
// exact arithmetic this equals n sweeps of Alg. 5 on A u = g; in mixed precision
// every residual the smoother sees is a correction-sized quantity, so the outer
// FP64 residual drives the iteration (iterative refinement).
static int was_block(Ctx& c, int l, double* u, int n, bool zero_start, bool want_res) {
  LevelHost& H = c.lv[l];
  const int prec = c.prm.precision;
  const size_t esz = prec == DGFAS_FP64 ? sizeof(double) : sizeof(float);
  if (zero_start) CK(cudaMemsetAsync(H.delta, 0, H.ndof * esz, c.stream));
  for (int s = 0; s < n; ++s) {
    if (s == 0 && zero_start) {
      if (prec == DGFAS_FP64) {
        CK(cudaMemcpyAsync(c.rw, H.r, H.ndof * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
      } else {
        RET(launch_to_float(c, H.r, (float*)c.rw, H.ndof));
      }
    } else {
      RET(launch_apply_corr(c, l, prec, H.delta, H.r, c.rw, 0));
    }
    RET(schwarz_into_delta(c, l));
  }
  if (want_res) RET(launch_apply_corr(c, l, prec, H.delta, H.r, H.r, 1));
  return launch_add_delta(c, H.ndof, prec, H.delta, u);
}

// Smoothing of A u = g on level l with lv[l].r = g - A u on entry.  With
// want_res, lv[l].r = g - A u of the smoothed u on exit.  zero_start = false
// means lv[l].delta holds a prolongated correction not yet added to u.
static int smooth(Ctx& c, int l, double* u, const double* g, int n, bool zero_start,
                  bool want_res) {
  if (c.prm.smoother == DGFAS_SCG) {
    if (c.prm.precision != DGFAS_FP64)   // correction form, as WAS (see scg_run)
      return scg_run(c, l, u, n, 0.0, c.prm.precision, !zero_start, want_res);
    if (!zero_start) {   // add the pending correction, then recompute the residual
      RET(launch_add_delta(c, c.lv[l].ndof, c.prm.precision, c.lv[l].delta, u));
      RET(launch_apply(c, l, DGFAS_FP64, u, g, c.lv[l].r, -1.0));
    }
    RET(scg_run(c, l, u, n, 0.0, c.prm.precision));
    if (want_res) RET(launch_apply(c, l, DGFAS_FP64, u, g, c.lv[l].r, -1.0));
    return DGFAS_OK;
  }
  if (n <= 0) {
    if (!zero_start) RET(launch_add_delta(c, c.lv[l].ndof, c.prm.precision, c.lv[l].delta, u));
    if (want_res && !zero_start) RET(launch_apply(c, l, DGFAS_FP64, u, g, c.lv[l].r, -1.0));
    return DGFAS_OK;
  }
  return was_block(c, l, u, n, zero_start, want_res);
}

// Root solve of lv[0] (A u_0 = g_0, g_0 in lv[0].gv): the dense inverse, or
// FP64 SCG (Alg. 6 as the coarse solver) from the current lv[0].u (the
// projection ubar_0 in a V-cycle) or from zero (zero_start).
static int root_solve(Ctx& c, bool zero_start) {
  if (c.prm.coarse != DGFAS_COARSE_SCG) return launch_root(c);
  LevelHost& R = c.lv[0];
  if (zero_start) CK(cudaMemsetAsync(R.u, 0, R.ndof * sizeof(double), c.stream));
  RET(launch_apply(c, 0, DGFAS_FP64, R.u, R.gv, R.r, -1.0));
  // FP64 iteration; in a mixed-precision context the Schwarz preconditioner
  // of the root runs in FP32 (it only shapes the search directions)
  const int pc = c.prm.precision == DGFAS_FP64 ? DGFAS_FP64 : DGFAS_FP32;
  return scg_run(c, 0, R.u, c.prm.root_steps, c.prm.root_rtol, pc, false, false, true);
}

// ---------------------------------------------------------------- FAS V-cycle
// Alg. 2 below the top level: lv[L].r holds the top residual of uL (after the
// top pre-smoothing).  Ends with the top correction I (u_{L-1} - P u_L) in
// lv[L].delta, not yet added to uL (the caller's top smoothing adds it).
static int down_up(Ctx& c, double* uL, const double* fL, int top = -1) {
  // top: the level that acts as the top (default: the finest); levels below
  // it keep their state in lv[l].u / lv[l].gv
  const int L = top < 0 ? (int)c.lv.size() - 1 : top;
  const int prec = c.prm.precision;
  for (int l = L; l >= 1; --l) {
    double* ul = l == L ? uL : c.lv[l].u;
    const double* gl = l == L ? fL : c.lv[l].gv;
    if (l < L) {
      // u_l is the projection ubar_l and g_l = A_l ubar_l + R r_{l+1}, so the
      // residual g_l - A_l u_l is R r_{l+1} (in lv[l].t) up to rounding; only
      // leaf rows (g = f) and frozen rows need the operator
      if (!c.lv[l].has_leaf && !c.lv[l].has_frozen)
        CK(cudaMemcpyAsync(c.lv[l].r, c.lv[l].t, c.lv[l].ndof * sizeof(double),
                           cudaMemcpyDeviceToDevice, c.stream));
      else
        RET(launch_apply(c, l, DGFAS_FP64, ul, gl, c.lv[l].r, -1.0));
      RET(smooth(c, l, ul, gl, c.prm.s1, true, true));
    }
    RET(launch_project(c, l, ul));                                   // u_{l-1} = P u_l
    RET(launch_restrict(c, l, c.lv[l].r, c.lv[l - 1].t));           // R r_l
    // the parent right-hand side g_{l-1} = A ubar_{l-1} + R r_l (tau correction).
    // Smoothing on an all-twig level below the top starts from its residual
    // R r_l and runs in correction form (WAS, and SCG in FP32 / BF16), so it
    // never reads g: the FP64 operator is needed only for the root, levels
    // with leaf or frozen rows, and the FP64 SCG smoother (residual from g)
    const LevelHost& P = c.lv[l - 1];
    if (l - 1 == 0 || P.has_leaf || P.has_frozen ||
        (c.prm.smoother == DGFAS_SCG && prec == DGFAS_FP64))
      RET(launch_apply(c, l - 1, DGFAS_FP64, P.u, P.t, P.gv, 1.0));
    if (P.has_leaf) RET(launch_leaf_rhs(c, l - 1, P.fl, P.gv));
  }
  RET(root_solve(c, false));
  for (int l = 1; l <= L; ++l) {
    double* ul = l == L ? uL : c.lv[l].u;
    const double* gl = l == L ? fL : c.lv[l].gv;
    RET(launch_prolong(c, l, ul, prec, c.lv[l].delta));             // delta_l = I (u_{l-1} - ubar)
    // the frozen update changed u^f, and with it the residual of the active rows:
    // the smoothing that follows starts from the residual of the updated u
    if (c.lv[l].has_frozen) RET(launch_apply(c, l, DGFAS_FP64, ul, gl, c.lv[l].r, -1.0));
    if (l < L) {
      // the post-smoothing starts from the residual of the pre-smoothed u_l,
      // which is still in lv[l].r (restriction only read it)
      RET(smooth(c, l, ul, gl, c.prm.s2, false, false));
    }
  }
  return DGFAS_OK;
}

// Alg. 2 on the top level: residual, s1 pre-sweeps, down/up legs, s2 post-sweeps.
// c.red receives the partial sums of |r|^2 of the residual after pre-smoothing.
static int vcycle_body(Ctx& c, double* u, const double* f) {
  const int L = (int)c.lv.size() - 1;
  RET(launch_apply(c, L, DGFAS_FP64, u, f, c.lv[L].r, -1.0));
  RET(smooth(c, L, u, f, c.prm.s1, true, true));
  RET(launch_sumsq(c, c.lv[L].r, c.lv[L].ndof, c.red));
  if (L == 0) return DGFAS_OK;
  RET(down_up(c, u, f));
  return smooth(c, L, u, f, c.prm.s2, false, false);
}

// One cycle of the crossover solve: down/up legs from the top residual in
// lv[L].r, n_sc top sweeps starting from the prolongated correction, FP64
// top residual and its partial sums (the stopping test of the next cycle).
static int solve_cycle_body(Ctx& c, double* u, const double* f) {
  const int L = (int)c.lv.size() - 1;
  RET(down_up(c, u, f));
  RET(smooth(c, L, u, f, c.prm.sc, false, false));
  RET(launch_apply(c, L, DGFAS_FP64, u, f, c.lv[L].r, -1.0));
  return launch_sumsq(c, c.lv[L].r, c.lv[L].ndof, c.red);
}

// Alg. 2 with level T < L as the top (u_T = lv[T].u, RHS f_T): the V-cycle
// of the full multigrid startup on the sub-hierarchy 0..T.
static int vcycle_sub(Ctx& c, int T, const double* fT) {
  double* uT = c.lv[T].u;
  RET(launch_apply(c, T, DGFAS_FP64, uT, fT, c.lv[T].r, -1.0));
  RET(smooth(c, T, uT, fT, c.prm.s1, true, true));
  RET(down_up(c, uT, fT, T));
  return smooth(c, T, uT, fT, c.prm.s2, false, false);
}

// u = I (u_c) on level l from lv[l-1].u: the solution interpolation of the
// full multigrid startup (the correction prolongation with a zero projection)
static int interpolate_solution(Ctx& c, int l, double* ul) {
  LevelHost& C = c.lv[l - 1];
  LevelHost& F = c.lv[l];
  // with ubar = 0 the prolongation writes I u_c into delta on active elements
  // and into u on frozen ones (delta = 0 there): u = 0, then u += delta
  CK(cudaMemsetAsync(C.ubar, 0, C.ndof * sizeof(double), c.stream));
  CK(cudaMemsetAsync(ul, 0, F.ndof * sizeof(double), c.stream));
  RET(launch_prolong(c, l, ul, DGFAS_FP64, F.delta));
  return launch_add_delta(c, F.ndof, DGFAS_FP64, F.delta, ul);
}

static bool graph_ok(Ctx& c) { return c.use_graph != 0; }

// Runs one cycle body on the caller's stream, or replays it as a CUDA graph
// captured on the context's internal stream (ordered after and before the
// caller's stream by events).
void drop_graphs(Ctx& c) {
  for (auto& g : c.graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = Ctx::GraphEntry{};
  }
}

static int run_body(Ctx& c, int kind, double* u, const double* f) {
  if (!graph_ok(c)) return kind == 0 ? vcycle_body(c, u, f) : solve_cycle_body(c, u, f);
  cudaStream_t user = c.stream;
  CK(cudaEventRecord(c.ev_in, user));
  CK(cudaStreamWaitEvent(c.cap, c.ev_in, 0));
  c.stream = c.cap;
  int rc = DGFAS_OK;
  Ctx::GraphEntry* hit = nullptr;
  for (auto& g : c.graphs)
    if (g.exec && g.u == u && g.f == f && g.kind == kind) hit = &g;
  if (!hit) {
    // the slot to (re)fill: an empty one, else the least recently used
    Ctx::GraphEntry* slot = &c.graphs[0];
    for (auto& g : c.graphs) {
      if (!g.exec) { slot = &g; break; }
      if (g.used < slot->used) slot = &g;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = Ctx::GraphEntry{};
    // this call's cycle runs uncaptured (it also sets the kernels' attributes) ...
    rc = kind == 0 ? vcycle_body(c, u, f) : solve_cycle_body(c, u, f);
    if (rc == DGFAS_OK && cudaStreamSynchronize(c.cap) != cudaSuccess) rc = DGFAS_ERR_CUDA;
    // ... then the same launches are captured for the following calls
    if (rc == DGFAS_OK) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = DGFAS_ERR_CUDA;
      } else {
        const long long k0 = g_kernels.load();
        int rc2 = kind == 0 ? vcycle_body(c, u, f) : solve_cycle_body(c, u, f);
        cudaError_t ce = cudaStreamEndCapture(c.cap, &g);
        slot->kernels = g_kernels.load() - k0;   // captured, not executed
        g_kernels -= slot->kernels;
        if (rc2 != DGFAS_OK) rc = rc2;
        else if (ce != cudaSuccess || cudaGraphInstantiate(&slot->exec, g, 0) != cudaSuccess) {
          set_error("graph capture/instantiate failed");
          rc = DGFAS_ERR_CUDA;
          slot->exec = nullptr;
        }
        if (g) cudaGraphDestroy(g);
        if (rc == DGFAS_OK) {
          slot->u = u;
          slot->f = f;
          slot->kind = kind;
          slot->used = ++c.graph_clock;
        }
      }
    }
  } else if (cudaGraphLaunch(hit->exec, c.cap) != cudaSuccess) {
    set_error("graph launch failed");
    rc = DGFAS_ERR_CUDA;
  } else {
    g_kernels += hit->kernels;
    hit->used = ++c.graph_clock;
  }
  c.stream = user;
  CK(cudaEventRecord(c.ev_out, c.cap));
  CK(cudaStreamWaitEvent(user, c.ev_out, 0));
  return rc;
}

// r_2 of Sec. 6.1: Euclidean norm of the residual over the leaf elements of
// all levels (synchronizes).  The top level's residual goes to lv[L].r.
static int composite_norm(Ctx& c, double* u, const double* f, double* out) {
  const int L = (int)c.lv.size() - 1;
  double s = 0.0;
  // the composite solution: twigs take the projection of the finer level
  // (top down, Eq. (6b)); frozen elements keep their interpolated values
  for (int l = L; l >= 1; --l) RET(launch_project(c, l, l == L ? u : c.lv[l].u));
  for (int l = 0; l <= L; ++l) {
    LevelHost& H = c.lv[l];
    if (!H.has_leaf) continue;
    const double* ul = l == L ? u : H.u;
    const double* gl = l == L ? f : H.fl;
    double* r = l == L ? H.r : H.t;
    RET(launch_apply(c, l, DGFAS_FP64, ul, gl, r, -1.0));
    RET(launch_sumsq_leaf(c, l, r, c.red));
    CK(cudaMemcpyAsync(c.red_host, c.red, c.red_blocks * sizeof(double), cudaMemcpyDeviceToHost,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (int i = 0; i < c.red_blocks; ++i) s += c.red_host[i];
  }
  *out = std::sqrt(s);
  return DGFAS_OK;
}

static double host_norm(Ctx& c) {
  double s = 0.0;
  for (int i = 0; i < c.red_blocks; ++i) s += c.red_host[i];
  return std::sqrt(s);
}

// ---------------------------------------------------------------- ABI
extern "C" long long dgfas_level_ndof(void* ctx, int level) {
  Ctx* c = (Ctx*)ctx;
  if (!c || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  return c->lv[level].ndof;
}

extern "C" int dgfas_node_coords(void* ctx, int level, double* xyz) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !xyz || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  return launch_node_coords(*c, level, xyz);
}

extern "C" int dgfas_assemble_rhs(void* ctx, const double* f, const double* uD, double* b) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !f || !b) return DGFAS_ERR_INVALID;
  return launch_rhs(*c, (int)c->lv.size() - 1, f, uD, b);
}

extern "C" int dgfas_assemble_rhs_level(void* ctx, int level, const double* f, const double* uD,
                                        double* b) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !f || !b || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  return launch_rhs(*c, level, f, uD, b);
}

extern "C" int dgfas_fmg(void* ctx, const double* const* f_levels, int cycles_per_level,
                         double* u_top) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !f_levels || !u_top || cycles_per_level < 1) return DGFAS_ERR_INVALID;
  const int L = (int)c->lv.size() - 1;
  for (int l = 0; l <= L; ++l)
    if (!f_levels[l]) return DGFAS_ERR_INVALID;
  if (L < 1) {
    set_error("fmg: needs at least two levels");
    return DGFAS_ERR_UNSUPPORTED;
  }
  // level 0: the V-cycle on the root alone is its exact solve
  CK(cudaMemcpyAsync(c->lv[0].gv, f_levels[0], c->lv[0].ndof * sizeof(double),
                     cudaMemcpyDeviceToDevice, c->stream));
  RET(root_solve(*c, true));
  for (int l = 1; l < L; ++l) {
    RET(interpolate_solution(*c, l, c->lv[l].u));
    for (int k = 0; k < cycles_per_level; ++k) RET(vcycle_sub(*c, l, f_levels[l]));
  }
  return interpolate_solution(*c, L, u_top);
}

extern "C" int dgfas_cmg(void* ctx, const double* const* f_levels, int n_sc, double* u_top) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !f_levels || !u_top || n_sc < 0) return DGFAS_ERR_INVALID;
  const int L = (int)c->lv.size() - 1;
  for (int l = 0; l <= L; ++l)
    if (!f_levels[l]) return DGFAS_ERR_INVALID;
  if (L < 1) {
    set_error("cmg: needs at least two levels");
    return DGFAS_ERR_UNSUPPORTED;
  }
  CK(cudaMemcpyAsync(c->lv[0].gv, f_levels[0], c->lv[0].ndof * sizeof(double),
                     cudaMemcpyDeviceToDevice, c->stream));
  RET(root_solve(*c, true));
  for (int l = 1; l < L; ++l) {
    LevelHost& H = c->lv[l];
    RET(interpolate_solution(*c, l, H.u));
    if (n_sc > 0) {
      // the smoothers start from the residual f_l - A_l u_l in lv[l].r
      RET(launch_apply(*c, l, DGFAS_FP64, H.u, f_levels[l], H.r, -1.0));
      RET(smooth(*c, l, H.u, f_levels[l], n_sc, true, false));
    }
  }
  return interpolate_solution(*c, L, u_top);
}

extern "C" int dgfas_element_energy(void* ctx, int level, const double* eps, double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !eps || !out || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  double* Ae = (double*)c->rw;   // scratch of at least the level's ndof doubles
  RET(launch_apply(*c, level, DGFAS_FP64, eps, nullptr, Ae, 1.0));
  return launch_element_dot(*c, level, eps, Ae, out);
}

extern "C" int dgfas_set_level_rhs(void* ctx, int level, const double* f) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !f || level < 0 || level >= (int)c->lv.size() - 1) return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  if (!H.fl) return DGFAS_OK;   // no leaf elements on this level: nothing to keep
  CK(cudaMemcpyAsync(H.fl, f, H.ndof * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return DGFAS_OK;
}

extern "C" int dgfas_composite_residual(void* ctx, double* u_top, const double* f_top,
                                        double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u_top || !f_top || !out) return DGFAS_ERR_INVALID;
  return composite_norm(*c, u_top, f_top, out);
}

extern "C" int dgfas_get_level_solution(void* ctx, int level, double* u) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || level < 0 || level >= (int)c->lv.size() - 1) return DGFAS_ERR_INVALID;
  CK(cudaMemcpyAsync(u, c->lv[level].u, c->lv[level].ndof * sizeof(double),
                     cudaMemcpyDeviceToDevice, c->stream));
  return DGFAS_OK;
}

extern "C" int dgfas_apply_op(void* ctx, int level, const double* u, const double* g, double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !out || u == out || level < 0 || level >= (int)c->lv.size()) {
    set_error("apply_op: invalid argument");
    return DGFAS_ERR_INVALID;
  }
  return g ? launch_apply(*c, level, DGFAS_FP64, u, g, out, -1.0)
           : launch_apply(*c, level, DGFAS_FP64, u, nullptr, out, 1.0);
}

extern "C" int dgfas_apply_op32(void* ctx, int level, const float* u, const double* g,
                                float* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !out || (const void*)u == (const void*)out || level < 0 ||
      level >= (int)c->lv.size()) {
    set_error("apply_op32: invalid argument");
    return DGFAS_ERR_INVALID;
  }
  return g ? launch_apply_corr(*c, level, DGFAS_FP32, u, g, out, 0)
           : launch_apply32(*c, level, u, out);
}

extern "C" int dgfas_schwarz_smooth(void* ctx, int level, double* u, const double* g, int n) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !g || n < 0 || level < 1 || level >= (int)c->lv.size()) {
    set_error("schwarz_smooth: invalid argument (levels >= 1 have a smoother)");
    return DGFAS_ERR_INVALID;
  }
  RET(launch_apply(*c, level, DGFAS_FP64, u, g, c->lv[level].r, -1.0));
  return smooth(*c, level, u, g, n, true, false);
}

extern "C" int dgfas_norm(void* ctx, int level, const double* v, double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !v || !out || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  return norm_dev(*c, v, c->lv[level].ndof, out);
}

extern "C" int dgfas_fas_vcycle(void* ctx, double* u, const double* f, double* rnorm) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !f) return DGFAS_ERR_INVALID;
  RET(run_body(*c, 0, u, f));
  if (rnorm) {
    CK(cudaMemcpyAsync(c->red_host, c->red, c->red_blocks * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *rnorm = host_norm(*c);
  }
  return DGFAS_OK;
}

extern "C" int dgfas_solve(void* ctx, double* u, const double* f, double rtol, int max_cycles,
                           dgfas_info* info) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !f || !(rtol > 0)) return DGFAS_ERR_INVALID;
  if (max_cycles <= 0) max_cycles = c->prm.max_cycles > 0 ? c->prm.max_cycles : 50;
  const int L = (int)c->lv.size() - 1;
  auto t0 = std::chrono::steady_clock::now();
  double r0;
  if (c->local) {
    RET(composite_norm(*c, u, f, &r0));
  } else {
    RET(launch_apply(*c, L, DGFAS_FP64, u, f, c->lv[L].r, -1.0));
    RET(norm_dev(*c, c->lv[L].r, c->lv[L].ndof, &r0));
  }
  RET(smooth(*c, L, u, f, c->prm.s1, true, false));
  RET(launch_apply(*c, L, DGFAS_FP64, u, f, c->lv[L].r, -1.0));
  int cycles = 0, rc = DGFAS_ERR_NOT_CONVERGED;
  double r = r0;
  if (info) { info->r0 = r0; memset(info->history, 0, sizeof(info->history)); }
  if (!(r0 > 0)) rc = (r0 == 0) ? DGFAS_OK : DGFAS_ERR_DIVERGED;
  while (rc == DGFAS_ERR_NOT_CONVERGED && cycles < max_cycles && L > 0) {
    RET(run_body(*c, 1, u, f));
    if (c->local) {
      RET(composite_norm(*c, u, f, &r));
      // the next cycle starts from the top residual (composite_norm left it in lv[L].r)
    } else {
      CK(cudaMemcpyAsync(c->red_host, c->red, c->red_blocks * sizeof(double),
                         cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      r = host_norm(*c);
    }
    if (info && cycles < 128) info->history[cycles] = r;
    ++cycles;
    if (!std::isfinite(r) || r > 1e3 * r0) rc = DGFAS_ERR_DIVERGED;
    else if (r <= rtol * r0) rc = DGFAS_OK;
  }
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->cycles = cycles;
    info->r_final = r;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  return rc;
}

// 1 if a tensor-core FD wait ran out since setup (then the patch is not valid)
extern "C" int dgfas_tc_error(void* ctx) {
  Ctx* c = (Ctx*)ctx;
  if (!c) return DGFAS_ERR_INVALID;
  int h = 0;
  if (cudaMemcpy(&h, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DGFAS_ERR_CUDA;
  return h;
}

extern "C" int dgfas_set_surrogate(void* ctx, int level, const double* g) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !g || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  const size_t n = 4 * (size_t)H.ne;
  CK(cudaMemcpyAsync(H.d_g, g, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  std::vector<double> tmp(n);
  CK(cudaMemcpyAsync(tmp.data(), H.d_g, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<float> f(tmp.begin(), tmp.end());
  CK(cudaMemcpy(H.f_g, f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  return DGFAS_OK;
}

extern "C" int dgfas_get_surrogate(void* ctx, int level, double* g) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !g || level < 0 || level >= (int)c->lv.size()) return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  CK(cudaMemcpyAsync(g, H.d_g, 4 * (size_t)H.ne * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return DGFAS_OK;
}

extern "C" int dgfas_use_graph(void* ctx, int enable) {
  Ctx* c = (Ctx*)ctx;
  if (!c) return DGFAS_ERR_INVALID;
  c->use_graph = enable ? 1 : 0;
  if (!enable) drop_graphs(*c);
  return DGFAS_OK;
}

// ---------------------------------------------------------------- autotuner
// field of Tune that `kernel` (0..3) selects
static int* tune_field(LevelHost& H, int kernel) {
  switch (kernel) {
    case 0: return &H.tune.apply64;
    case 1: return &H.tune.apply32;
    case 2: return &H.tune.fd;
    case 3: return &H.tune.fdtc;
  }
  return nullptr;
}

// one launch of the tunable `kernel` on level l on scratch data
static int tune_run(Ctx& c, int l, int kernel) {
  LevelHost& H = c.lv[l];
  const int prec = c.prm.precision;
  if (kernel == 0) return launch_apply(c, l, DGFAS_FP64, H.delta, nullptr, H.r, 1.0);
  if (kernel == 1) return launch_apply_corr(c, l, prec, H.delta, H.r, c.rw, 0);
  return launch_fd(c, l, prec, c.rw);
}

extern "C" int dgfas_autotune(void* ctx, int reps, double* report, int max_entries,
                              int* n_entries) {
  Ctx* c = (Ctx*)ctx;
  if (!c || reps <= 0 || (max_entries > 0 && !report)) return DGFAS_ERR_INVALID;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int n_rep = 0, rc = DGFAS_OK;
  for (int l = 0; l < (int)c->lv.size() && rc == DGFAS_OK; ++l) {
    LevelHost& H = c->lv[l];
    // the scratch operands: level work vectors (their contents are rebuilt at
    // the start of every smoothing block and cycle)
    CK(cudaMemsetAsync(H.delta, 0, H.ndof * sizeof(double), c->stream));
    CK(cudaMemsetAsync(H.r, 0, H.ndof * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->rw, 0, H.ndof * sizeof(double), c->stream));
    for (int k = 0; k < 4 && rc == DGFAS_OK; ++k) {
      if (l == 0 && k > 0) continue;   // the root level is not smoothed
      int cand[16];
      const int nc = tune_candidates(*c, l, k, cand + 1, 15);
      if (nc == 0) continue;
      cand[0] = 0;   // the built-in default
      int* field = tune_field(H, k);
      double best = 1e300, t_def = 0.0;
      int best_v = 0;
      for (int i = 0; i <= nc && rc == DGFAS_OK; ++i) {
        *field = cand[i];
        rc = tune_run(*c, l, k);   // warm-up (and first-use attributes)
        if (rc != DGFAS_OK) break;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) { rc = DGFAS_ERR_CUDA; break; }
        for (int q = 0; q < reps && rc == DGFAS_OK; ++q) rc = tune_run(*c, l, k);
        if (rc != DGFAS_OK) break;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) { rc = DGFAS_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double t = ms / reps;
        if (i == 0) t_def = t;
        if (t < best) { best = t; best_v = cand[i]; }
      }
      *field = best_v;
      if (rc == DGFAS_OK && n_rep < max_entries) {
        double* r5 = report + 5 * n_rep;
        r5[0] = l; r5[1] = k; r5[2] = best_v; r5[3] = best; r5[4] = t_def;
      }
      if (rc == DGFAS_OK) ++n_rep;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // launch shapes are baked into a captured graph: capture again on next use
  drop_graphs(*c);
  if (n_entries) *n_entries = n_rep;
  return rc;
}

extern "C" int dgfas_set_tuning(void* ctx, int level, int kernel, int value) {
  Ctx* c = (Ctx*)ctx;
  if (!c || level < 0 || level >= (int)c->lv.size() || kernel < 0 || kernel > 3) {
    set_error("set_tuning: invalid argument");
    return DGFAS_ERR_INVALID;
  }
  if (value != 0) {
    int cand[16];
    const int nc = tune_candidates(*c, level, kernel, cand, 16);
    bool ok = false;
    for (int i = 0; i < nc; ++i) ok |= cand[i] == value;
    if (!ok) {
      set_error("set_tuning: value is not a candidate launch shape of this kernel and level");
      return DGFAS_ERR_INVALID;
    }
  }
  *tune_field(c->lv[level], kernel) = value;
  drop_graphs(*c);
  return DGFAS_OK;
}

extern "C" int dgfas_get_tuning(void* ctx, int level, int kernel, int* value, int* candidates,
                                int max_candidates, int* n_candidates) {
  Ctx* c = (Ctx*)ctx;
  if (!c || level < 0 || level >= (int)c->lv.size() || kernel < 0 || kernel > 3 || !value)
    return DGFAS_ERR_INVALID;
  *value = *tune_field(c->lv[level], kernel);
  if (n_candidates) {
    int cand[16];
    const int nc = tune_candidates(*c, level, kernel, cand, 16);
    for (int i = 0; i < nc && i < max_candidates && candidates; ++i) candidates[i] = cand[i];
    *n_candidates = nc;
  }
  return DGFAS_OK;
}

extern "C" const char* dgfas_strerror(int code) {
  switch (code) {
    case DGFAS_OK: return "ok";
    case DGFAS_ERR_INVALID: return "invalid argument";
    case DGFAS_ERR_OOM: return "device out of memory";
    case DGFAS_ERR_CUDA: return "CUDA runtime error";
    case DGFAS_ERR_MESH: return "invalid mesh (non-positive Jacobian or indefinite root)";
    case DGFAS_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case DGFAS_ERR_DIVERGED: return "diverged (NaN/Inf or residual growth)";
    case DGFAS_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown error";
}

extern "C" const char* dgfas_last_error(void) { return g_err.c_str(); }

// Host-only view of one fast-diagonalization variant (no device work): the
// subdomain width n, S [n][n] (row = node, column = mode), lambda [n], W [n].
extern "C" int dgfas_host_fd_variant(int p, double delta, double mu_star, int variant, double* S,
                                     double* lam, double* W, int* n_out) {
  if (p < 1 || p > 10 || variant < 0 || variant > 15 || !S || !lam || !W || !n_out ||
      !(delta > 0 && delta < 0.5))
    return DGFAS_ERR_INVALID;
  const int m = host::overlap_layers(p, delta);
  const char sc[4] = {'i', 'd', 'n', 'f'};
  std::vector<double> Sv, lv, wv;
  host::fd_variant(p, m, mu_star, delta, sc[variant / 4], sc[variant % 4], Sv, lv, wv);
  const int n = (int)lv.size();
  *n_out = n;
  for (int i = 0; i < n * n; ++i) S[i] = Sv[i];
  for (int i = 0; i < n; ++i) { lam[i] = lv[i]; W[i] = wv[i]; }
  return DGFAS_OK;
}

// Per-kernel timing of the smoother on `level` with CUDA events on the
// context's stream: `reps` sweeps; ms_out[0..3] = average duration of the
// smoother-precision residual of the correction, the FD kernel, the combine
// kernel and the FP64 residual apply.  u is not modified.
extern "C" int dgfas_profile_sweep(void* ctx, int level, double* u, const double* g, int reps,
                                   double* ms_out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !u || !g || !ms_out || reps <= 0 || level < 1 || level >= (int)c->lv.size())
    return DGFAS_ERR_INVALID;
  LevelHost& H = c->lv[level];
  const int prec = c->prm.precision;
  const size_t esz = prec == DGFAS_FP64 ? sizeof(double) : sizeof(float);
  cudaEvent_t ev[5];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double acc[4] = {0, 0, 0, 0};
  RET(launch_apply(*c, level, DGFAS_FP64, u, g, H.r, -1.0));
  CK(cudaMemsetAsync(H.delta, 0, H.ndof * esz, c->stream));
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(ev[0], c->stream));
    RET(launch_apply_corr(*c, level, prec, H.delta, H.r, c->rw, 0));
    CK(cudaEventRecord(ev[1], c->stream));
    RET(launch_fd(*c, level, prec, c->rw));
    CK(cudaEventRecord(ev[2], c->stream));
    RET(launch_combine(*c, level, prec, H.delta));
    CK(cudaEventRecord(ev[3], c->stream));
    RET(launch_apply(*c, level, DGFAS_FP64, u, g, c->lv[level].t ? c->lv[level].t : H.r, -1.0));
    CK(cudaEventRecord(ev[4], c->stream));
    CK(cudaEventSynchronize(ev[4]));
    for (int k = 0; k < 4; ++k) {
      float ms;
      CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
      acc[k] += ms;
    }
  }
  for (int k = 0; k < 4; ++k) ms_out[k] = acc[k] / reps;
  for (auto& e : ev) cudaEventDestroy(e);
  return DGFAS_OK;
}

int launch_fma_peak(cudaStream_t st, int fp64, int iters, double* tflops);

// Measured FMA throughput (TFLOP/s) of this GPU in FP64 and FP32: the ALU roofline.
extern "C" int dgfas_fma_peak(double* tflops_fp64, double* tflops_fp32) {
  if (!tflops_fp64 || !tflops_fp32) return DGFAS_ERR_INVALID;
  RET(launch_fma_peak(nullptr, 1, 4096, tflops_fp64));
  return launch_fma_peak(nullptr, 0, 65536, tflops_fp32);
}

// Number of kernels this library has launched in the process so far, the
// kernel nodes of replayed CUDA graphs included.
extern "C" long long dgfas_kernel_launches(void) { return g_kernels.load(); }
