// Internal structures shared by the host setup, the kernels and the driver.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgfas.h"

#define DGFAS_MAX_N 11     // p <= 10
#define DGFAS_MAX_NS 16    // subdomain width per direction

// Per-level device view passed by value to kernels.
template <typename T>
struct LevelView {
  int ne, N, m, nsm;          // elements, nodes per direction, overlap layers, max subdomain width
  int box;                    // 1: every element is an axis-aligned box (factors from h)
  T nu, kappa;
  const int* nbr;             // [ne][6]
  const int* nbr27;           // [ne][27]
  const signed char* cls;     // [ne]
  const T* h;                 // [ne][3] box widths (box levels)
  const T* bx;                // [ne][6] box factors g_d, a_d (box levels)
  const T* Lhat;              // [N][N] D^T W D
  const T* G;                 // [ne][6][N^3] volume metric (general levels)
  const T* fW;                // [ne][6][N^2] face quadrature weights (general)
  const T* fc;                // [ne][6][3][N^2] W n . grad xi_t (general)
  const T* mu;                // [ne][6] face penalty
  const T* mass;              // [ne][N^3] lumped mass (kappa != 0, general) or null
  const T* tri;               // [ne][24] trilinear map x = a0 + a1 xi + a2 eta + a3 zeta
                              // + a4 xi eta + a5 xi zeta + a6 eta zeta + a7 xi eta zeta:
                              // a1..a7 (x, y, z each) and 3 pad (general levels)
  const void* coff;           // [ne][27] combine offsets (int, or long long when
                              // ne NS^3 >= 2^31): patch index of the element's node
                              // (0,0,0) in neighbour slot s's patch, or the minimum
  const T* D;                 // [N][N]
  const T* w;                 // [N] GLL weights
  const T* x;                 // [N] GLL nodes
  // Schwarz
  const unsigned char* var;   // [ne][3] variant 4*left+right per direction (side types
                              // 0 interior, 1 Dirichlet, 2 Neumann, 3 frozen neighbour)
  const T* g;                 // [ne][4] surrogate coefficients g0..g3
  const T* S;                 // [16][nsm][nsm]  S[v][row][col]
  const T* lam;               // [16][nsm]
  const T* W;                 // [16][nsm]
  const uint4* Btc;           // [16][2][32] BF16 operand tiles S^T and S (tensor-core FD)
};

struct TransferView {
  int nef, nec, Nf, Nc, h;    // h: 1 for h-refinement (8 children)
  int cs;                     // p-transfer whose matrices are centrosymmetric (even-odd kernels)
  const int* parent;          // [nef]
  const int* octant;          // [nef]
  const int* children;        // [nec][8] (-1 none); p-refinement: children[E][0] = E
  const signed char* clsf;    // [nef] fine classes
  const double* I;            // [2][Nf][Nc]
  const double* P;            // [2][Nc][Nf]
};

// Launch shapes chosen by the autotuner (0 = the built-in default):
// elements per CTA of the FP64 and smoother-precision box operators and of
// the narrow-subdomain FD kernel, CTAs per SM of the tensor-core FD kernel.
// largest root level solved by its dense inverse (n^2 doubles, 512 MB at 8192)
#define DGFAS_MAX_ROOT 8192

struct Tune {
  int apply64 = 0, apply32 = 0, fd = 0, fdtc = 0;
};

struct LevelHost {
  int p, N, ne, m, nsm, box;
  long long ndof;
  std::vector<int> nbr, nbr27, parent, octant;
  std::vector<signed char> cls;
  std::vector<double> corners;
  // device arrays (FP64 and FP32 copies of the geometry / tables)
  int *d_nbr = nullptr, *d_nbr27 = nullptr, *d_parent = nullptr, *d_octant = nullptr,
      *d_children = nullptr;
  signed char* d_cls = nullptr;
  unsigned char* d_var = nullptr;
  double *d_bx = nullptr, *d_Lhat = nullptr;
  float *f_bx = nullptr, *f_Lhat = nullptr;
  double *d_h = nullptr, *d_G = nullptr, *d_fW = nullptr, *d_fc = nullptr, *d_mu = nullptr,
         *d_mass = nullptr, *d_D = nullptr, *d_w = nullptr, *d_g = nullptr, *d_S = nullptr,
         *d_lam = nullptr, *d_W = nullptr, *d_x = nullptr;
  float *f_h = nullptr, *f_G = nullptr, *f_fW = nullptr, *f_fc = nullptr, *f_mu = nullptr,
        *f_mass = nullptr, *f_D = nullptr, *f_w = nullptr, *f_g = nullptr, *f_S = nullptr,
        *f_lam = nullptr, *f_W = nullptr, *f_x = nullptr;
  double* d_tri = nullptr;
  float* f_tri = nullptr;
  int* d_coff32 = nullptr;          // combine offsets (one of the two)
  long long* d_coff64 = nullptr;
  bool coff32 = true;
  uint4* d_Btc = nullptr;                  // BF16 FD operand tiles per variant
  double *d_I = nullptr, *d_P = nullptr;   // transfer from level-1 to this level
  // work vectors
  double *u = nullptr, *gv = nullptr, *r = nullptr, *ubar = nullptr, *t = nullptr;
  double* delta = nullptr;   // smoother correction (FP64 or FP32 storage)
  double* fl = nullptr;      // RHS of the leaf elements (levels below the top)
  int has_leaf = 0, has_frozen = 0;
  LevelView<double> v64;
  LevelView<float> v32;
  TransferView tr;
  Tune tune;
};

struct Ctx;
void drop_graphs(Ctx& c);   // destroys every captured cycle body

struct Ctx {
  cudaStream_t stream = nullptr;
  dgfas_params prm{};
  double nu = 1.0, kappa = 0.0;
  std::vector<LevelHost> lv;
  // scratch
  void* patch = nullptr;        // Schwarz patch buffer (max over levels)
  size_t patch_bytes = 0;
  void* rw = nullptr;           // smoother working residual (smoother precision)
  cudaStream_t cap = nullptr;   // internal stream for graph capture / replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int red_blocks = 0;           // CTAs of the reductions: 4 per SM of the device
  double* red = nullptr;        // reduction partials [5 * red_blocks + 64]: norms use
                                // [0, G), SCG's scalar products [G, 5G) (2G CTAs, two
                                // sums each), G = red_blocks
  double* red_host = nullptr;   // pinned
  double* scg_buf = nullptr;    // SCG vectors (p, q, z, r0) for the largest level
  double* apply_scratch = nullptr;   // two-pass FP64 curvilinear operator: F [e][3][N^3]
  size_t apply_scratch_n = 0;        // and face data [e][6][2][N^2] of the largest level
  double* dscal = nullptr;      // device scalars of the SCG recurrences
  int* dcnt = nullptr;          // ticket counters of the single-pass reductions
  int* tc_err = nullptr;        // set by the tensor-core FD kernel when a wait ran out
  double* Ainv = nullptr;       // root inverse
  int n_root = 0;
  // graphs
  int use_graph = 0;
  // captured cycle bodies, one per (u, f, kind) in use (a caller that
  // alternates buffers, e.g. to overlap its copies with the solve, replays
  // each without capturing again); least recently used entry replaced
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    const double* u = nullptr;
    const double* f = nullptr;
    int kind = -1;
    long long kernels = 0;       // kernel nodes of the captured graph
    unsigned long long used = 0;
  };
  static constexpr int kGraphs = 4;
  GraphEntry graphs[kGraphs];
  unsigned long long graph_clock = 0;
  int local = 0;                 // leaves below the top or frozen elements exist
};

// kernels.cu
int launch_apply(Ctx& c, int l, int prec, const double* u, const double* b, void* out,
                 double alpha);
int launch_apply_corr(Ctx& c, int l, int prec, const void* delta, const double* b, void* out,
                      int out_fp64);
int launch_fd(Ctx& c, int l, int prec, const void* r);
int launch_fd_tc(Ctx& c, int l, const float* r);
// candidate launch shapes of the tunable kernels of level l (autotuner)
int tune_candidates(Ctx& c, int l, int kernel, int* out, int max_out);
int launch_combine(Ctx& c, int l, int prec, void* delta);
int launch_add_delta(Ctx& c, long long n, int prec, const void* d, double* u);
int launch_combine_to(Ctx& c, int l, int prec, double* z);
int launch_combine_to32(Ctx& c, int l, float* z);
int launch_apply32(Ctx& c, int l, const float* u, float* out);
int prepare_transfer(const TransferView& T);          // set-up: kernel attributes
int launch_project(Ctx& c, int l, const double* uf);   // lv[l-1].u = ubar = P uf
int launch_restrict(Ctx& c, int l, const double* rf, double* rc);
int launch_prolong(Ctx& c, int l, double* uf, int prec, void* delta);  // delta = I (u_c - ubar)
int launch_root(Ctx& c);
// set-up of the dense root inverse
int launch_identity(Ctx& c, double* E, int n);
int launch_element_dot(Ctx& c, int l, const double* a, const double* b, double* out);
int launch_root_inverse(Ctx& c, double* A, int n, double shift, double* work, int* flag);
int launch_sumsq(Ctx& c, const double* v, long long n, double* partial_out);
int launch_dot(Ctx& c, const double* a, const double* b, long long n, double* partial_out);
int launch_axpy(Ctx& c, long long n, double alpha, const double* x, double* y);
int launch_node_coords(Ctx& c, int l, double* xyz);
int launch_rhs(Ctx& c, int l, const double* f, const double* uD, double* b);
int launch_sumsq_leaf(Ctx& c, int l, const double* v, double* part);
int launch_leaf_rhs(Ctx& c, int l, const double* f, double* g);
int launch_to_float(Ctx& c, const double* x, float* y, long long n);
// scg.cu: Alg. 6 with device-resident scalars (no host synchronization);
// the SCG work buffer holds 4 FP64 (or 5 FP32) vectors of the largest level,
// each followed by kScgPad doubles of padding
constexpr long long kScgPad = 768;
int scg_run(Ctx& c, int l, double* u, int n, double rtol, int prec, bool pending = false,
            bool want_res = false, bool fp64_vectors = false);
extern std::atomic<long long> g_kernels;   // kernels launched (graph replays included)

void set_error(const std::string& s);
