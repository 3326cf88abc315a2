// Host side of the C ABI declared in include/fdtd.h.
//
// Device data layout: every one of the six components is stored in the same
// padded box of (nz+1) planes x (ny+1) rows x pitch elements, pitch a
// multiple of 32 elements (128-byte aligned rows for FP32).  Sample (i, j, k)
// of any component lives at k*plane + j*pitch + i; entries outside the
// component's compact Yee shape are zero and never written.  Node j of a
// grid line and face j of the paired H component share an element offset,
// which is what lets one kernel walk both.
//
// The hot loop is in line_kernels.cuh; this file holds validation, FP64
// coefficient precompute, the scheme schedules (Sec. II) and the launches.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "adjoint_kernels.cuh"
#include "aux_kernels.cuh"
#include "line_kernels.cuh"
#include "line4_kernels.cuh"

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);

enum { EX = 0, EY, EZ, HX, HY, HZ };
enum { AX_X = 0, AX_Y = 1, AX_Z = 2 };

struct PairGeom {
  int ec = 0, hc = 0, axis = 0, sign = 0, N = 0;
  bool rows = false;
  long long ls = 0, os = 0, os2 = 0;
  int lane_lo = 0, lane_hi = 0, o_lo = 0, n_o = 0, o2_lo = 0, n_o2 = 0;
  long long n_lines() const {
    return rows ? (long long)n_o * n_o2 : (long long)std::max(0, lane_hi - lane_lo) * n_o;
  }
  bool empty() const { return N < 2 || n_lines() <= 0; }
};

// Coefficients of one pair for one procedure length h.
struct PairCoef {
  double kb = 0, kd = 0;  // signed s*b/d_eta, s*d/d_eta
  void* tab = nullptr;    // uniform media: [12][tlen] hi/lo rows (1/beta, m, c, PF, PB, kappa g) in T
  int tlen = 0;
  int L = 16;             // segment length the carry-product rows are built for
  int jc = 1 << 30;       // uniform media: first converged segment start
  double cv[6] = {0, 0, 0, 0, 0, 0};  // converged (hi, lo) of 1/beta, m, c
  bool wall_fix = false;  // uniform media: the rank-one wall correction rows are built
  int kg_len = 0;         // the correction is zero from this node on (a multiple of L)
  double qf[2][32] = {{0}}, qb[2][32] = {{0}};
  int jc4 = 1 << 30, je4 = -1;  // fourth order: nodes whose factor rows all equal cv4
  double cv4[14] = {0};
  void* nq = nullptr;     // per-node media (field layout, T): 1/|b_j|
  void* nib = nullptr;    //   1/beta_j (hi)
  void* nibl = nullptr;   //   1/beta_j (lo, FP32 only)
  double ks = 0, offh = 0, offl = 0;  // per-node: scaled-row coupling, off-diagonal
  void* nkd = nullptr;    // per-node mu: H coupling of each face (field layout, T)
  void* noffh = nullptr;  //   off-diagonal of each face, hi
  void* noffl = nullptr;  //   off-diagonal of each face, lo (FP32 only)
};

struct StridedCfg {
  bool ok = false;
  int lanes = 32, L = 16;
};

struct ProcCoef {
  bool valid = false;
  int op = 0;  // 0 = A, 1 = B
  double h = 0;
  PairCoef pc[3];
};

}  // namespace

struct fdtd_s {
  fdtd_desc desc;
  int nx, ny, nz;
  double dx, dy, dz, dt;
  int scheme, prec;
  size_t esize;
  cudaStream_t stream;
  long long pitch, plane, count;
  void* f[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* scratch[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* stage = nullptr;  // contiguous staging buffer of host copies (one component)
  PairGeom geom[2][3];
  StridedCfg strided_cfg[2];  // y lines, z lines
  int num_sms = 0;
  int* d_err = nullptr;       // set by kernels whose bounded waits gave up
  bool use_tma = true;
  // TMA descriptors of the y/z line tiles, per component and box kind
  // TMA descriptors per component and box kind (0: y-line tiles, 1: z-line
  // tiles, 2: x-row tiles)
  CUtensorMap tmap[6][3];
  const void* tmap_ptr[6][3] = {{nullptr}};
  int tmap_bn[6][3] = {{0}};
  int tmap_lanes[6][3] = {{0}};
  // 0: A main, 1: B main, 2: B at dt/2 (FLOD2 processing); lossy media
  // only: 3, 4 = B at dt and at dt/2 with the loss term's sign flipped, the
  // matrices of the FADI output relation and of the FLOD2 output processing
  // (procedures of negative length, whose loss diagonal changes sign while
  // the second-difference part does not)
  ProcCoef proc[5];
  bool per_node = false;
  bool shape_tuned = false;   // per-node y/z launch shapes chosen by timing
  double eps_r = 1.0, mu_r = 1.0;          // uniform media
  double* eps_node[3] = {nullptr, nullptr, nullptr};  // per-node eps_r at E samples (device)
  std::vector<double> eps_host[3];  // the same on the host, only while coefficients are built
  // lossy media: electric conductivity sigma [S/m]; the loss -sigma/eps E is
  // split evenly between A and B, so each procedure of length h adds
  // b sigma / 4 to the implicit diagonal (a host-side change of the pivots)
  bool lossy = false;
  double sigma_u = 0.0;             // uniform sigma (when sig_node is null)
  // order of the spatial differences: 2 (Yee) or 4 (fourth-order staggered,
  // PEC images; uniform lossless media, single grids)
  int order = 2;
  void* tmp4 = nullptr;             // order 4: field-shaped scratch of the line solves, one
                                    // per E component (pairs of a procedure run concurrently)
  void* yseq = nullptr;             // FP64 y/z lines solved one thread per line: the forward
                                    // values, one field-shaped array per E component
  double* sig_node[3] = {nullptr, nullptr, nullptr};  // per-node sigma at E samples (device)
  std::vector<double> sig_host[3];  // the same on the host, only while coefficients are built
  bool mu_var = false;              // per-node mu (general media kernels)
  double* mu_node[3] = {nullptr, nullptr, nullptr};   // per-face mu_r at H samples (device)
  std::vector<double> mu_host[3];   // the same on the host, only while coefficients are built
  bool poisoned = false;
  bool pending_init = true;   // FADI/FLOD2: state holds the physical field
  bool output_valid = false;  // scratch holds the physical field of this step
  long long steps = 0;
  // source
  int src_comp = -1, src_i = 0, src_j = 0, src_k = 0;
  std::vector<double> src_current;
  double src_scale = 0;  // f_E = src_scale * I
  // probes
  int nprobes = 0;
  int probe_comp[fdtd::kMaxProbes];
  long long probe_at[fdtd::kMaxProbes];
  long long probe_start[fdtd::kMaxProbes];
  double* d_probe = nullptr;   // [kMaxProbes][probe_cap]
  double* d_stash = nullptr;
  long long probe_cap = 0;
  double* d_partial = nullptr;
  int partial_n = 0;
  // reference value of the scheme invariant (out[1] of fdtd_energy), taken
  // on the device right after (re)initialisation of a run with no source;
  // fdtd_energy reports FDTD_ERR_UNSTABLE when the invariant grows past it
  bool inv_dirty = true;        // take a new reference at the next step
  bool inv_have = false;        // d_ref_partial holds a reference
  double inv_ref = -1.0;        // its value once read back (< 0: not yet)
  double* d_ref_partial = nullptr;
  // accounting
  long long launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;     // reusable events
  // one-step CUDA graph (steps without probes or per-launch timing): the
  // three pairs of each procedure on parallel branches
  cudaStream_t g_run = nullptr, g_br[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t g_in = nullptr, g_out = nullptr, g_fork = nullptr, g_join[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t g_exec = nullptr;
  std::vector<const void*> g_bound;     // state pointers the graph was captured with
  long long g_kernels = 0;              // kernels per replay
  double* d_srcval = nullptr;           // f_E(n) = src_scale * I(n), n < src_current.size()
  long long srcval_len = 0;
  long long* d_step = nullptr;          // step index read by graph-replayed source kernels
  std::vector<std::pair<int, std::pair<int, int>>> ev_rec;  // (class, (start ev, stop ev))
  long long timed_launches[3] = {0, 0, 0};
  double timed_ms[3] = {0, 0, 0};
  double bytes_per_launch[3] = {0, 0, 0};
};

namespace {

int single_tune(fdtd_t* h);

// NVTX range over a scope: host-side annotations for profilers (ncu's
// --nvtx filters); without a tool attached the calls return at once.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

// Every device allocation of the library goes through dev_malloc.  A test
// hook (fdtd_debug_fail_alloc) can make the n-th next one fail as an
// out-of-memory would, without calling CUDA, to exercise the error paths.
std::atomic<long long> g_fail_alloc_in{-1};

cudaError_t dev_malloc(void** p, size_t n) {
  long long k = g_fail_alloc_in.load();
  while (k >= 0) {
    if (g_fail_alloc_in.compare_exchange_weak(k, k == 0 ? -1 : k - 1)) {
      if (k == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, n);
}

int cuda_fail(fdtd_t* h, cudaError_t e) {
  if (e == cudaSuccess) return FDTD_OK;
  if (h) h->poisoned = true;
  fprintf(stderr, "fdtd: CUDA error: %s\n", cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_fail(h, _e);       \
  } while (0)

void comp_extent(int c, int nx, int ny, int nz, int* sx, int* sy, int* sz) {
  switch (c) {
    case EX: *sx = nx; *sy = ny + 1; *sz = nz + 1; break;
    case EY: *sx = nx + 1; *sy = ny; *sz = nz + 1; break;
    case EZ: *sx = nx + 1; *sy = ny + 1; *sz = nz; break;
    case HX: *sx = nx + 1; *sy = ny; *sz = nz; break;
    case HY: *sx = nx; *sy = ny + 1; *sz = nz; break;
    default: *sx = nx; *sy = ny; *sz = nz + 1; break;
  }
}

// The three (E, H, axis, sign) pairs of A (Eq. 33) and B (Eq. 34).
void build_geometry(fdtd_t* h) {
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  const int E_[2][3] = {{EX, EY, EZ}, {EX, EY, EZ}};
  const int H_[2][3] = {{HZ, HX, HY}, {HY, HZ, HX}};
  const int A_[2][3] = {{AX_Y, AX_Z, AX_X}, {AX_Z, AX_X, AX_Y}};
  for (int op = 0; op < 2; ++op) {
    for (int q = 0; q < 3; ++q) {
      PairGeom g;
      g.ec = E_[op][q];
      g.hc = H_[op][q];
      g.axis = A_[op][q];
      g.sign = op == 0 ? +1 : -1;
      g.rows = g.axis == AX_X;
      g.N = g.axis == AX_X ? nx : (g.axis == AX_Y ? ny : nz);
      // x range of lines (strided) and the other transverse ranges:
      // tangential E on a wall is not an unknown, so those lines are skipped.
      if (g.axis == AX_X) {
        g.ls = 1;
        g.os = h->pitch;
        g.os2 = h->plane;
        if (g.ec == EY) {  // Ey lines (j, k): j in [0, ny), k in [1, nz-1]
          g.o_lo = 0; g.n_o = ny; g.o2_lo = 1; g.n_o2 = nz - 1;
        } else {           // Ez lines: j in [1, ny-1], k in [0, nz)
          g.o_lo = 1; g.n_o = ny - 1; g.o2_lo = 0; g.n_o2 = nz;
        }
      } else if (g.axis == AX_Y) {
        g.ls = h->pitch;
        g.os = h->plane;
        if (g.ec == EX) {  // Ex lines (i, k): i in [0, nx), k in [1, nz-1]
          g.lane_lo = 0; g.lane_hi = nx; g.o_lo = 1; g.n_o = nz - 1;
        } else {           // Ez lines (i, k): i in [1, nx-1], k in [0, nz)
          g.lane_lo = 1; g.lane_hi = nx; g.o_lo = 0; g.n_o = nz;
        }
      } else {
        g.ls = h->plane;
        g.os = h->pitch;
        if (g.ec == EX) {  // Ex lines (i, j): i in [0, nx), j in [1, ny-1]
          g.lane_lo = 0; g.lane_hi = nx; g.o_lo = 1; g.n_o = ny - 1;
        } else {           // Ey lines (i, j): i in [1, nx-1], j in [0, ny)
          g.lane_lo = 1; g.lane_hi = nx; g.o_lo = 0; g.n_o = ny;
        }
      }
      if (g.n_o < 0) g.n_o = 0;
      if (g.n_o2 < 0) g.n_o2 = 0;
      h->geom[op][q] = g;
    }
  }
}

// nodes per lane of the x-line kernel: the smallest instantiated L with 32 L >= N
int pick_rows_L(int N) {
  static const int kL[] = {1, 2, 4, 8, 12, 16, 24, 32};
  const int need = (N + 31) / 32;
  for (int L : kL)
    if (L >= need) return L;
  return -1;
}

// FP64 fields on uniform media, pairs of at least this many lines: the solve
// is bound by the FP64 pipe, so every lane reads the coefficient tables
// (PairParams::tables_only) and x lines of 32 < N <= 256 take 16 nodes on 4,
// 8 or 16 lanes (proc_rows_lpl_kernel).  Smaller pairs are bound by latency,
// where the converged constants (no loads) and short per-lane chains win.
constexpr long long kFp64ThroughputLines = 4096;

bool fp64_throughput_pair(const fdtd_t* h, const PairGeom& g) {
  return h->prec == FDTD_F64 && !h->per_node && g.n_lines() >= kFp64ThroughputLines;
}

// Nodes per lane (L) and lanes per line of a pair's x lines: the shape above,
// else one warp per line with the smallest L that covers the line.  The
// uniform-media coefficient tables are built for this L.
int rows_lanes(const fdtd_t* h, const PairGeom& g) {
  if (!fp64_throughput_pair(h, g) || g.N <= 32 || g.N > 256) return 32;
  return g.N <= 64 ? 4 : (g.N <= 128 ? 8 : 16);
}
int rows_L(const fdtd_t* h, const PairGeom& g) { return rows_lanes(h, g) < 32 ? 16 : pick_rows_L(g.N); }

// segments per line for a block of LANES-wide segments: ceil(N / L) rounded
// up so that the block is a whole number of warps (extra segments lie past
// the line end and hold zeros)
int segments(int N, int L, int lanes) {
  const int P = (N + L - 1) / L;
  const int m = 32 / lanes;
  return ((P + m - 1) / m) * m;
}

double spacing(const fdtd_t* h, int axis) { return axis == AX_X ? h->dx : (axis == AX_Y ? h->dy : h->dz); }

template <typename T>
int upload(fdtd_t* h, void** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.size());
  for (size_t q = 0; q < src.size(); ++q) tmp[q] = (T)src[q];
  if (!*dst) CK(dev_malloc((void**)dst, tmp.size() * sizeof(T)));
  CK(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FDTD_OK;
}

int upload_any(fdtd_t* h, void** dst, const std::vector<double>& src) {
  return h->prec == FDTD_F64 ? upload<double>(h, dst, src) : upload<float>(h, dst, src);
}

void free_coef(ProcCoef& pc) {
  for (auto& c : pc.pc) {
    if (c.tab) cudaFree(c.tab);
    if (c.nq) cudaFree(c.nq);
    if (c.nib) cudaFree(c.nib);
    if (c.nibl) cudaFree(c.nibl);
    if (c.nkd) cudaFree(c.nkd);
    if (c.noffh) cudaFree(c.noffh);
    if (c.noffl) cudaFree(c.noffl);
    c = PairCoef();
  }
  pc.valid = false;
}

// eps_r at every E sample: mean of the in-domain cells sharing the edge.
// mu_r at the H samples of component c (HX, HY, HZ): the mean of the two
// cells sharing the face (cells outside the domain skipped).
void face_mu(const fdtd_t* h, const double* mr, int c, std::vector<double>& out) {
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  out.assign((size_t)h->count, 1.0);
  int sx, sy, sz;
  comp_extent(c, nx, ny, nz, &sx, &sy, &sz);
  for (int k = 0; k < sz; ++k)
    for (int j = 0; j < sy; ++j)
      for (int i = 0; i < sx; ++i) {
        double s = 0;
        int n = 0;
        for (int a = -1; a <= 0; ++a) {
          int ci = i, cj = j, ck = k;
          if (c == HX) ci = i + a;   // Hx (i, j+1/2, k+1/2): cells (i-1..i, j, k)
          if (c == HY) cj = j + a;   // Hy (i+1/2, j, k+1/2): cells (i, j-1..j, k)
          if (c == HZ) ck = k + a;   // Hz (i+1/2, j+1/2, k): cells (i, j, k-1..k)
          if (ci < 0 || cj < 0 || ck < 0 || ci >= nx || cj >= ny || ck >= nz) continue;
          s += mr[((size_t)ck * ny + cj) * nx + ci];
          ++n;
        }
        out[(size_t)k * h->plane + (size_t)j * h->pitch + i] = n ? s / n : 1.0;
      }
}

void edge_eps(const fdtd_t* h, const double* er, int c, std::vector<double>& out) {
  const int nx = h->nx, ny = h->ny, nz = h->nz;
  out.assign((size_t)h->count, 0.0);
  int sx, sy, sz;
  comp_extent(c, nx, ny, nz, &sx, &sy, &sz);
  for (int k = 0; k < sz; ++k)
    for (int j = 0; j < sy; ++j)
      for (int i = 0; i < sx; ++i) {
        double s = 0;
        int n = 0;
        for (int a = -1; a <= 0; ++a)
          for (int b = -1; b <= 0; ++b) {
            int ci = i, cj = j, ck = k;
            if (c == EX) { cj = j + a; ck = k + b; }
            if (c == EY) { ci = i + a; ck = k + b; }
            if (c == EZ) { ci = i + a; cj = j + b; }
            if (ci < 0 || cj < 0 || ck < 0 || ci >= nx || cj >= ny || ck >= nz) continue;
            s += er[((size_t)ck * ny + cj) * nx + ci];
            ++n;
          }
        out[(size_t)k * h->plane + (size_t)j * h->pitch + i] = n ? s / n : 1.0;
      }
}

// lines of at most this many cells take the block-tiled fourth-order kernel
constexpr int kLine4TileMaxN = 512;

// Fourth-order differences: the banded LU (bandwidth 3, no pivoting: the
// matrix is symmetric positive definite) of one pair's line system
//   1/2 w - (kb kd / 2) D'(D' w) = r   on the interior nodes 1..N-1,
// D' the stencil (c1 = 9/8, c2 = -1/24 as the kernel rounds it) with PEC
// images, formed in FP64 from the couplings the kernel uses.  Rows (hi, lo)
// of fdtd::T4_*: multipliers l1..l3 of L, 1/u0 and u1..u3 of U per node.
int build_pair4(fdtd_t* h, const PairGeom& g, PairCoef& c, double hh) {
  const bool f32 = h->prec == FDTD_F32;
  auto rnd = [&](double x) { return f32 ? (double)(float)x : x; };
  const double de = spacing(h, g.axis);
  const double b = hh / (2.0 * kEps0 * h->eps_r);
  c.kb = rnd(g.sign * b / de);
  c.kd = rnd(c.kd);
  const double bd = c.kb * c.kd;
  const double c1 = 1.125, c2 = rnd(-1.0 / 24.0);
  const int N = std::max(g.N, 1);
  const int n = std::max(N - 1, 0);   // unknowns: nodes 1..N-1
  // stencils with images: (D' E)_f over node offsets, (D' H)_j over faces
  auto face_img = [&](int f) { return f < 0 ? -1 - f : (f > N - 1 ? 2 * N - 1 - f : f); };
  // dense band of K = D'_HE D'_EH: row k (node k+1), columns k-3..k+3
  std::vector<double> band((size_t)n * 7, 0.0);
  auto addK = [&](int row, int col, double v) {
    if (col < 0 || col >= n) return;  // a wall node: fixed at zero
    const int o = col - row;
    if (o < -3 || o > 3) return;
    band[(size_t)row * 7 + (o + 3)] += v;
  };
  const int fo[4] = {0, -1, 1, -2};
  const double fw[4] = {c1, -c1, c2, -c2};
  const int no[4] = {1, 0, 2, -1};
  const double nw[4] = {c1, -c1, c2, -c2};
  for (int k = 0; k < n; ++k) {
    const int j = k + 1;
    for (int a = 0; a < 4; ++a) {
      const int f = face_img(j + fo[a]);
      for (int q = 0; q < 4; ++q) {
        int m = f + no[q];
        double sgn = 1.0;
        if (m < 0) { m = -m; sgn = -1.0; }
        if (m > N) { m = 2 * N - m; sgn = -1.0; }
        addK(k, m - 1, fw[a] * sgn * nw[q]);
      }
    }
  }
  // M = 1/2 I - (bd/2) K, factored in place (band storage, offsets -3..3)
  for (int k = 0; k < n; ++k) {
    for (int o = 0; o < 7; ++o) band[(size_t)k * 7 + o] *= -0.5 * bd;
    band[(size_t)k * 7 + 3] += 0.5;
  }
  auto at = [&](int r, int col) -> double& { return band[(size_t)r * 7 + (col - r + 3)]; };
  for (int i = 0; i < n; ++i) {
    const double piv = at(i, i);
    if (!(std::fabs(piv) > 0)) return FDTD_ERR_INVALID_ARG;
    for (int k = i + 1; k <= std::min(i + 3, n - 1); ++k) {
      const double l = at(k, i) / piv;
      at(k, i) = l;
      for (int m = i + 1; m <= std::min(i + 3, n - 1); ++m) at(k, m) -= l * at(i, m);
    }
  }
  c.tlen = ((N + 4 + 31) / 32) * 32;
  const int tl = c.tlen;
  auto hi = [&](double x) { return f32 ? (double)(float)x : x; };
  auto lo = [&](double x) { return f32 ? (double)(float)(x - (double)(float)x) : 0.0; };
  std::vector<double> tab((size_t)fdtd::T4_ROWS * tl, 0.0);
  auto put = [&](int row, int j, double v) {
    tab[(size_t)row * tl + j] = hi(v);
    tab[(size_t)(row + 1) * tl + j] = lo(v);
  };
  for (int k = 0; k < n; ++k) {
    const int j = k + 1;
    if (k >= 1) put(fdtd::T4_L1H, j, at(k, k - 1));
    if (k >= 2) put(fdtd::T4_L2H, j, at(k, k - 2));
    if (k >= 3) put(fdtd::T4_L3H, j, at(k, k - 3));
    put(fdtd::T4_IUH, j, 1.0 / at(k, k));
    if (k + 1 < n) put(fdtd::T4_U1H, j, at(k, k + 1));
    if (k + 2 < n) put(fdtd::T4_U2H, j, at(k, k + 2));
    if (k + 3 < n) put(fdtd::T4_U3H, j, at(k, k + 3));
  }
  // Away from the walls the factor rows of a homogeneous line converge: find
  // the run of nodes around the middle whose rows (as stored, hi and lo) all
  // equal the middle node's, which the tiled kernel's sweeps then take from
  // registers instead of the table.
  c.jc4 = 1 << 30;
  c.je4 = -1;
  if (N >= 16) {
    const int jm = N / 2;
    auto same = [&](int j) {
      for (int r = 0; r < fdtd::T4_ROWS; ++r)
        if (tab[(size_t)r * tl + j] != tab[(size_t)r * tl + jm]) return false;
      return true;
    };
    int a = jm, b = jm;
    while (a - 1 >= 1 && same(a - 1)) --a;
    while (b + 1 <= N - 1 && same(b + 1)) ++b;
    c.jc4 = a;
    c.je4 = b;
    for (int r = 0; r < fdtd::T4_ROWS; ++r) c.cv4[r] = tab[(size_t)r * tl + jm];
  }
  c.jc = 1 << 30;
  c.wall_fix = false;
  return upload_any(h, &c.tab, tab);
}

// FP64 factorisation of the line systems of one procedure (operator op,
// length hh):  1/2 w_j - (b_j/2)(d/d^2)(w_{j+1} - 2 w_j + w_{j-1}) = r_j, plus
// loss_sign * b_j sigma_j / 4 on the diagonal in lossy media (loss_sign = -1
// for the matrices of procedures run with negative length).
int build_proc(fdtd_t* h, int slot, int op, double hh, double loss_sign = 1.0) {
  ProcCoef& P = h->proc[slot];
  free_coef(P);
  P.op = op;
  P.h = hh;
  for (int q = 0; q < 3; ++q) {
    const PairGeom& g = h->geom[op][q];
    PairCoef& c = P.pc[q];
    const double de = spacing(h, g.axis);
    const double d = hh / (2.0 * kMu0 * h->mu_r);
    c.kd = g.sign * d / de;
    if (h->order == 4) {
      int rc = build_pair4(h, g, c, hh);
      if (rc) return rc;
      continue;
    }
    if (!h->per_node) {
      const double b = hh / (2.0 * kEps0 * h->eps_r);
      c.kb = g.sign * b / de;
      // Factor the system the kernel actually applies: with FP32 couplings
      // kb, kd the line operator is 1/2 - (kb kd / 2) (second difference), so
      // form b d / d_eta^2 from the rounded couplings.  The procedure is then
      // an exact Cayley transform of a (1e-8-perturbed) skew operator and
      // keeps its energy invariant instead of drifting.
      double bd = b * d / (de * de);
      if (h->prec == FDTD_F32) {
        c.kb = (double)(float)c.kb;
        c.kd = (double)(float)c.kd;
        bd = c.kb * c.kd;
      }
      const double off = -bd / 2.0;
      const double diag = 0.5 + bd + (h->lossy ? loss_sign * b * h->sigma_u / 4.0 : 0.0);
      const int N = std::max(g.N, 1);
      const int L = g.rows ? std::max(1, rows_L(h, g)) : h->strided_cfg[g.axis == AX_Y ? 0 : 1].L;
      c.L = L;
      // covers every segment a kernel may form: P*L <= N + 4L - 1 with L <= 32
      c.tlen = ((std::max(N + 160, 32 * std::max(1, pick_rows_L(N))) + 31) / 32) * 32;
      const int tl = c.tlen;
      std::vector<double> ib(tl, 0.0), m(tl, 0.0), cc(tl, 0.0), pf(tl, 0.0), pb(tl, 0.0);
      for (int j = 1; j <= N - 1; ++j) {
        const double beta = (j == 1) ? diag : diag - off * off * ib[j - 1];
        ib[j] = 1.0 / beta;
      }
      for (int j = 0; j < tl; ++j) {
        m[j] = (j >= 1) ? off * ib[j - 1] : 0.0;
        cc[j] = off * ib[j];
      }
      // carry products within each segment [s L, s L + L)
      for (int j0 = 0; j0 + L <= tl; j0 += L) {
        double q = 1.0;
        for (int t = 0; t < L; ++t) { q *= -m[j0 + t]; pf[j0 + t] = q; }
        q = 1.0;
        for (int t = L - 1; t >= 0; --t) { q *= -cc[j0 + t]; pb[j0 + t] = q; }
      }
      const bool f32 = h->prec == FDTD_F32;
      auto hi = [&](double x) { return f32 ? (double)(float)x : x; };
      auto lo = [&](double x) { return f32 ? (double)(float)(x - (double)(float)x) : 0.0; };
      // The converged factors: the same recurrence continued until it stops
      // changing (a fixed point, or a 2-cycle in the last bit).  Long lines
      // reach these values in their tables; x lines use them on every lane
      // together with the rank-one wall correction below.
      double beta_inf = diag;
      for (int it = 0; it < 100000; ++it) {
        const double nb = diag - off * off * (1.0 / beta_inf);
        if (nb == beta_inf) break;
        beta_inf = nb;
      }
      const double ib_inf = 1.0 / beta_inf, mc_inf = off * ib_inf;
      // Rank-one wall correction kappa g_j: the constant factors are the LU
      // of T' = T + delta e_1 e_1^T with delta = beta_inf - diag; g solves
      // T' g = e_1 with them (nodes 1..N-1) and kappa = delta/(1 - delta g_1)
      std::vector<double> kg(tl, 0.0);
      if (N >= 2) {
        std::vector<double> yg((size_t)N + 1, 0.0), gg((size_t)N + 2, 0.0);
        for (int j = 1; j <= N - 1; ++j) yg[j] = (j == 1 ? 1.0 : 0.0) - (j > 1 ? mc_inf * yg[j - 1] : 0.0);
        for (int j = N - 1; j >= 1; --j) gg[j] = yg[j] * ib_inf - mc_inf * gg[j + 1];
        const double delta = beta_inf - diag;
        const double kappa = delta / (1.0 - delta * gg[1]);
        // terms below 2^-50 of w'_1 change no result: drop them, so that the
        // segments past the last nonzero term skip the correction
        int last = 0;
        for (int j = 1; j <= N - 1; ++j) {
          kg[j] = kappa * gg[j];
          if (std::fabs(kg[j]) < 0x1p-50) kg[j] = 0.0;
          else last = j;
        }
        c.kg_len = last > 0 ? ((last + 1 + L - 1) / L) * L : 0;
      }
      std::vector<double> tab((size_t)fdtd::TB_ROWS * tl, 0.0);
      const std::vector<double>* rows[6] = {&ib, &m, &cc, &pf, &pb, &kg};
      for (int r = 0; r < 6; ++r)
        for (int j = 0; j < tl; ++j) {
          tab[(size_t)(2 * r) * tl + j] = hi((*rows[r])[j]);
          tab[(size_t)(2 * r + 1) * tl + j] = lo((*rows[r])[j]);
        }
      // converged constants (hi, lo) and segment carry products; jc = first
      // segment start from which every full segment's table entries equal
      // them
      c.jc = 1 << 30;
      {
        const double cvv[3] = {ib_inf, mc_inf, mc_inf};
        for (int k = 0; k < 3; ++k) { c.cv[2 * k] = hi(cvv[k]); c.cv[2 * k + 1] = lo(cvv[k]); }
        double qf = 1.0;
        for (int t = 0; t < L; ++t) { qf *= -mc_inf; c.qf[0][t] = hi(qf); c.qf[1][t] = lo(qf); }
        double qb = 1.0;
        for (int t = L - 1; t >= 0; --t) { qb *= -mc_inf; c.qb[0][t] = hi(qb); c.qb[1][t] = lo(qb); }
      }
      c.wall_fix = L >= 2;
      const int last_seg = ((N) / L - 1) * L;  // start of the last segment with j0 + L <= N
      if (N >= 2 && last_seg >= 0) {
        auto seg_ok = [&](int j0) {
          for (int t = 0; t < L; ++t) {
            const int j = j0 + t;
            if (hi(ib[j]) != c.cv[0] || lo(ib[j]) != c.cv[1] || hi(m[j]) != c.cv[2] || lo(m[j]) != c.cv[3] ||
                hi(cc[j]) != c.cv[4] || lo(cc[j]) != c.cv[5] || hi(pf[j]) != c.qf[0][t] || lo(pf[j]) != c.qf[1][t] ||
                hi(pb[j]) != c.qb[0][t] || lo(pb[j]) != c.qb[1][t])
              return false;
          }
          return true;
        };
        int jc = last_seg;
        while (jc - L >= 0 && seg_ok(jc - L)) jc -= L;
        c.jc = seg_ok(last_seg) ? jc : (1 << 30);
      }
      int rc = upload_any(h, &c.tab, tab);
      if (rc) return rc;
    } else {
      // Per-node media: rows scaled by 1/b_j (a symmetric matrix),
      //   q_j w_j / 2 - (|ks| |kd| / 2) (w_{j+1} - 2 w_j + w_{j-1}) = q_j E_j + ks (H_j - H_{j-1}),
      // q_j = 1/|b_j|, ks = s sign(h) / d_eta.  Every line is factored in FP64
      // from exactly the q_j, ks, kd the kernel uses (rounded to the field
      // precision first), so each procedure is an exact Cayley transform of
      // the medium those rounded values describe.
      const bool f32 = h->prec == FDTD_F32;
      auto rnd = [&](double x) { return f32 ? (double)(float)x : x; };
      c.kd = rnd(c.kd);
      c.ks = rnd(g.sign * (hh >= 0 ? 1.0 : -1.0) / de);
      const double kk = std::fabs(c.ks) * std::fabs(c.kd);
      const double off = -kk / 2.0;
      c.offh = rnd(off);
      c.offl = f32 ? (double)(float)(off - c.offh) : 0.0;
      std::vector<double> nq((size_t)h->count, 0.0), nib((size_t)h->count, 0.0), nibl;
      if (f32) nibl.assign((size_t)h->count, 0.0);
      // per-node mu: each face f (between nodes f and f+1) has its own
      // coupling kd_f and off-diagonal -|ks| |kd_f| / 2
      std::vector<double> nkd, noffh, noffl;
      if (h->mu_var) {
        nkd.assign((size_t)h->count, 0.0);
        noffh.assign((size_t)h->count, 0.0);
        if (f32) noffl.assign((size_t)h->count, 0.0);
      }
      const double* mr = h->mu_var ? h->mu_host[g.hc - 3].data() : nullptr;
      const double* er = h->eps_host[g.ec].data();
      const double* sr = (h->lossy && !h->sig_host[g.ec].empty()) ? h->sig_host[g.ec].data() : nullptr;
      // scaled rows: the loss adds loss_sign * sigma_j / 4 to the diagonal
      auto loss_at = [&](long long at) {
        return h->lossy ? loss_sign * (sr ? sr[at] : h->sigma_u) / 4.0 : 0.0;
      };
      const long long nl = g.n_lines();
      for (long long line = 0; line < nl; ++line) {
        long long base;
        if (g.rows) {
          const int jo = g.o_lo + (int)(line % g.n_o);
          const int ko = g.o2_lo + (int)(line / g.n_o);
          base = (long long)ko * g.os2 + (long long)jo * g.os;
        } else {
          const int nlx = g.lane_hi - g.lane_lo;
          const int i = g.lane_lo + (int)(line % nlx);
          const int o = g.o_lo + (int)(line / nlx);
          base = (long long)o * g.os + i;
        }
        double ibm = 0;
        if (!h->mu_var) {
          for (int j = 1; j <= g.N - 1; ++j) {
            const long long at = base + (long long)j * g.ls;
            const double b = std::fabs(hh) / (2.0 * kEps0 * er[at]);
            const double q = rnd(1.0 / b);
            const double diag = q / 2.0 + kk + loss_at(at);
            const double beta = diag - off * off * ibm;
            const double ib = 1.0 / beta;
            nq[at] = q;
            nib[at] = rnd(ib);
            if (f32) nibl[at] = (double)(float)(ib - nib[at]);
            ibm = ib;
          }
          continue;
        }
        // kk_f = |ks| |kd_f| of the faces, from the kd_f the kernel uses
        std::vector<double> kkf((size_t)g.N, 0.0);
        for (int f = 0; f < g.N; ++f) {
          const long long at = base + (long long)f * g.ls;
          const double kdf = rnd(g.sign * (hh / (2.0 * kMu0 * mr[at])) / de);
          const double kkv = std::fabs(c.ks) * std::fabs(kdf);
          const double offf = -kkv / 2.0;
          kkf[(size_t)f] = kkv;
          nkd[at] = kdf;
          noffh[at] = rnd(offf);
          if (f32) noffl[at] = (double)(float)(offf - noffh[at]);
        }
        for (int j = 1; j <= g.N - 1; ++j) {
          const long long at = base + (long long)j * g.ls;
          const double b = std::fabs(hh) / (2.0 * kEps0 * er[at]);
          const double q = rnd(1.0 / b);
          const double diag = q / 2.0 + (kkf[(size_t)j] + kkf[(size_t)j - 1]) / 2.0 + loss_at(at);
          const double offm = -kkf[(size_t)j - 1] / 2.0;  // face j-1, between nodes j-1 and j
          const double beta = diag - offm * offm * ibm;
          const double ib = 1.0 / beta;
          nq[at] = q;
          nib[at] = rnd(ib);
          if (f32) nibl[at] = (double)(float)(ib - nib[at]);
          ibm = ib;
        }
      }
      int rc = upload_any(h, &c.nq, nq);
      if (rc) return rc;
      if ((rc = upload_any(h, &c.nib, nib))) return rc;
      if (f32 && (rc = upload_any(h, &c.nibl, nibl))) return rc;
      if (h->mu_var) {
        if ((rc = upload_any(h, &c.nkd, nkd))) return rc;
        if ((rc = upload_any(h, &c.noffh, noffh))) return rc;
        if (f32 && (rc = upload_any(h, &c.noffl, noffl))) return rc;
      }
    }
  }
  P.valid = true;
  return FDTD_OK;
}

int build_all_coefs(fdtd_t* h) {
  const double dt = h->dt;
  int rc;
  if (h->scheme == FDTD_FSS) {
    if ((rc = build_proc(h, 0, 0, dt / 2))) return rc;
    if ((rc = build_proc(h, 1, 1, dt))) return rc;
  } else {
    if ((rc = build_proc(h, 0, 0, dt))) return rc;
    if ((rc = build_proc(h, 1, 1, dt))) return rc;
  }
  if (h->scheme == FDTD_FLOD2) {
    if ((rc = build_proc(h, 2, 1, dt / 2))) return rc;
  } else {
    free_coef(h->proc[2]);
  }
  free_coef(h->proc[3]);
  free_coef(h->proc[4]);
  if (h->lossy && h->scheme == FDTD_FADI && (rc = build_proc(h, 3, 1, dt, -1.0))) return rc;
  if (h->lossy && h->scheme == FDTD_FLOD2 && (rc = build_proc(h, 4, 1, dt / 2, -1.0))) return rc;
  return FDTD_OK;
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------


template <typename T>
fdtd::PairParams<T> make_params(const fdtd_t* h, const PairGeom& g, const PairCoef& c, double sgn,
                                double alpha, double beta, double kd_mul, void* const* in,
                                void* const* out) {
  fdtd::PairParams<T> p;
  p.e_in = (const T*)in[g.ec];
  p.h_in = (const T*)in[g.hc];
  p.e_out = (T*)out[g.ec];
  p.h_out = (T*)out[g.hc];
  p.ls = g.ls;
  p.os = g.os;
  p.os2 = g.os2;
  p.lane_lo = g.lane_lo;
  p.lane_hi = g.lane_hi;
  p.o_lo = g.o_lo;
  p.n_o = g.n_o;
  p.o2_lo = g.o2_lo;
  p.n_o2 = g.n_o2;
  p.N = g.N;
  p.kb = (T)(sgn * c.kb);
  p.kd = (T)(sgn * kd_mul * c.kd);
  p.alpha = (T)alpha;
  p.beta = (T)beta;
  p.e_unit = (alpha == 1.0 && beta == -1.0) ? 1 : 0;
  p.tab = (const T*)c.tab;
  p.tlen = c.tlen;
  p.jc = c.jc;
  for (int k = 0; k < 6; ++k) p.cv[k] = (T)c.cv[k];
  for (int t = 0; t < 32; ++t) {
    p.qf[0][t] = (T)c.qf[0][t];
    p.qf[1][t] = (T)c.qf[1][t];
    p.qb[0][t] = (T)c.qb[0][t];
    p.qb[1][t] = (T)c.qb[1][t];
  }
  p.err = h->d_err;
  p.nq = (const T*)c.nq;
  p.nib = (const T*)c.nib;
  p.nibl = (const T*)c.nibl;
  p.ks = (T)(sgn * c.ks);
  p.offh = (T)c.offh;
  p.offl = (T)c.offl;
  p.d_out = nullptr;
  p.nkd = (const T*)c.nkd;
  p.noffh = (const T*)c.noffh;
  p.noffl = (const T*)c.noffl;
  p.kd_scale = (T)(sgn * kd_mul);
  p.n_elem = h->count;
  p.tables_only = fp64_throughput_pair(h, g) ? 1 : 0;
  // FP32 fields in homogeneous media: converged factors on every lane plus
  // the rank-one wall correction (tune[1] bit 7: the table lanes instead)
  p.wall_fix = (c.wall_fix && sizeof(T) == 4 && (h->desc.tune[1] & 128) == 0) ? 1 : 0;
  p.kg_len = c.kg_len;
  // one scratch array per E component: the three pairs of a procedure run
  // concurrently (graph branches) and each has its own E component
  p.tmp4 = h->tmp4 ? (T*)h->tmp4 + (size_t)g.ec * h->count : nullptr;
  p.c2_4 = (T)(-1.0 / 24.0);
  p.jc4 = c.jc4;
  p.je4 = c.je4;
  for (int k = 0; k < 14; ++k) p.cv4[k] = (T)c.cv4[k];
  return p;
}

template <typename T, int LANES, int L>
void launch_strided_L(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, bool per_node) {
  const int P = segments(g.N, L, LANES);
  dim3 grid((unsigned)((g.lane_hi + LANES - 1) / LANES), (unsigned)g.n_o);
  const int threads = P * LANES;
  const size_t smem = 6 * (size_t)(P | 1) * LANES * sizeof(T);
  if (per_node)
    fdtd::proc_strided_kernel<T, LANES, L, true><<<grid, threads, smem, h->stream>>>(p);
  else
    fdtd::proc_strided_kernel<T, LANES, L, false><<<grid, threads, smem, h->stream>>>(p);
}

template <typename T, int L>
void launch_rows_L(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, bool per_node) {
  const int wpb = 8;
  const long long nl = g.n_lines();
  const unsigned blocks = (unsigned)((nl + wpb - 1) / wpb);
  if (per_node)
    fdtd::proc_rows_kernel<T, L, true><<<blocks, wpb * 32, 0, h->stream>>>(p);
  else if (sizeof(T) == 4 && L >= 2 && p.wall_fix && g.N == 32 * L && (h->desc.tune[1] & 2048) == 0)
    fdtd::proc_rows_kernel<T, L, false, (sizeof(T) == 4 && L >= 2), (sizeof(T) == 4 && L >= 2)>
        <<<blocks, wpb * 32, 0, h->stream>>>(p);
  else if (sizeof(T) == 4 && L >= 2 && p.wall_fix)
    fdtd::proc_rows_kernel<T, L, false, (sizeof(T) == 4 && L >= 2)><<<blocks, wpb * 32, 0, h->stream>>>(p);
  else
    fdtd::proc_rows_kernel<T, L, false><<<blocks, wpb * 32, 0, h->stream>>>(p);
}

// x lines of FP64 uniform media: 16 nodes per lane, lanes lanes per line.
template <typename T>
void launch_rows_lpl(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, int lanes) {
  const int wpb = 8;
  const long long warps = (g.n_lines() * lanes + 31) / 32;
  const unsigned blocks = (unsigned)((warps + wpb - 1) / wpb);
  if (lanes == 4) fdtd::proc_rows_lpl_kernel<T, 16, 4><<<blocks, wpb * 32, 0, h->stream>>>(p);
  else if (lanes == 8) fdtd::proc_rows_lpl_kernel<T, 16, 8><<<blocks, wpb * 32, 0, h->stream>>>(p);
  else fdtd::proc_rows_lpl_kernel<T, 16, 16><<<blocks, wpb * 32, 0, h->stream>>>(p);
}

// (LANES, L) of the y/z line kernels.  A block holds every segment of LANES
// lines, so P * LANES threads with P = ceil(N / L); the choice must fit the
// register file (checked against the compiled kernel's attributes).
template <typename T, int LANES, int L>
const void* strided_fn(bool pn) {
  return pn ? (const void*)fdtd::proc_strided_kernel<T, LANES, L, true>
            : (const void*)fdtd::proc_strided_kernel<T, LANES, L, false>;
}

template <typename T>
const void* strided_fn_rt(bool pn, int lanes, int L) {
  if (lanes == 32 && L == 8) return strided_fn<T, 32, 8>(pn);
  if (lanes == 32 && L == 16) return strided_fn<T, 32, 16>(pn);
  if (lanes == 32 && L == 32) return strided_fn<T, 32, 32>(pn);
  if (lanes == 16 && L == 8) return strided_fn<T, 16, 8>(pn);
  if (lanes == 16 && L == 16) return strided_fn<T, 16, 16>(pn);
  if (lanes == 16 && L == 32) return strided_fn<T, 16, 32>(pn);
  if (lanes == 8 && L == 16) return strided_fn<T, 8, 16>(pn);
  if (lanes == 8 && L == 32) return strided_fn<T, 8, 32>(pn);
  return nullptr;
}

template <typename T>
void launch_strided(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, bool pn, int lanes, int L) {
  if (lanes == 32 && L == 8) launch_strided_L<T, 32, 8>(h, g, p, pn);
  else if (lanes == 32 && L == 16) launch_strided_L<T, 32, 16>(h, g, p, pn);
  else if (lanes == 32 && L == 32) launch_strided_L<T, 32, 32>(h, g, p, pn);
  else if (lanes == 16 && L == 8) launch_strided_L<T, 16, 8>(h, g, p, pn);
  else if (lanes == 16 && L == 16) launch_strided_L<T, 16, 16>(h, g, p, pn);
  else if (lanes == 16 && L == 32) launch_strided_L<T, 16, 32>(h, g, p, pn);
  else if (lanes == 8 && L == 16) launch_strided_L<T, 8, 16>(h, g, p, pn);
  else if (lanes == 8 && L == 32) launch_strided_L<T, 8, 32>(h, g, p, pn);
}

template <typename T>
StridedCfg choose_strided(int N, bool pn, int tune_L) {
  // preference order: widest rows first (coalescing), then the L that keeps
  // registers low enough for two or more resident blocks.
  static const int cand32[][2] = {{32, 16}, {32, 8}, {32, 32}, {16, 32}, {8, 32}, {8, 32}};
  static const int cand64[][2] = {{16, 16}, {16, 8}, {16, 32}, {8, 16}, {8, 32}, {8, 32}};
  const int(*cand)[2] = sizeof(T) == 8 ? cand64 : cand32;
  StridedCfg best;
  for (int pass = 0; pass < 2; ++pass) {
    for (int q = 0; q < 6; ++q) {
      const int lanes = cand[q][0], L = cand[q][1];
      if (pass == 0 && tune_L && L != tune_L) continue;
      const int P = segments(N, L, lanes);
      if (P > 32) continue;  // the carry chains scan at most 32 segments (one warp)
      const void* fn = strided_fn_rt<T>(pn, lanes, L);
      if (!fn) continue;
      cudaFuncAttributes a;
      if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) continue;
      if (P * lanes > a.maxThreadsPerBlock) continue;
      best.ok = true;
      best.lanes = lanes;
      best.L = L;
      return best;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// TMA-fed y/z line solves (homogeneous media, lines of at most 256 cells)
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// nodes per thread of the TMA kernel (the coefficient tables' carry
// products are built for the strided L, which must match)
template <typename T>
constexpr int tma_L() { return 16; }
int tma_L_rt(const fdtd_t*) { return 16; }


// FP32 fields only: in FP64 the direct-load kernel (16 lines x 16 nodes per
// thread, more resident warps) measured 14 % faster per step at 256^3 than
// the TMA-fed kernel, whose 8-line FP64 tiles keep 8 warps per SM.
bool tma_eligible(const fdtd_t* h, const PairGeom& g) {
  // the coefficient tables' carry products are built for the strided L
  return h->use_tma && h->prec == FDTD_F32 && !h->per_node && !g.rows && g.N >= 2 && g.N <= 256 &&
         h->strided_cfg[g.axis == AX_Y ? 0 : 1].L == tma_L_rt(h) && tensor_map_encoder() != nullptr;
}

// Tensor map of component c for tiles of LANES lines x BN nodes along y
// (kind 0) or z (kind 1), or of `lanes` rows x BN elements along x (kind 2).
// Re-encoded when the array moved.
int get_tmap(fdtd_t* h, int c, int kind, int BN, int lanes, const CUtensorMap** out) {
  if (h->tmap_ptr[c][kind] != h->f[c] || h->tmap_bn[c][kind] != BN || h->tmap_lanes[c][kind] != lanes) {
    cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)(h->ny + 1), (cuuint64_t)(h->nz + 1)};
    cuuint64_t strides[2] = {(cuuint64_t)h->pitch * h->esize, (cuuint64_t)h->plane * h->esize};
    cuuint32_t box[3] = {(cuuint32_t)lanes, kind == 0 ? (cuuint32_t)BN : 1u, kind == 0 ? 1u : (cuuint32_t)BN};
    if (kind == 2) {
      box[0] = (cuuint32_t)BN;
      box[1] = (cuuint32_t)lanes;
      box[2] = 1u;
    }
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = tensor_map_encoder()(&h->tmap[c][kind],
                                      h->prec == FDTD_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                      3, h->f[c], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      fprintf(stderr, "fdtd: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
      return FDTD_ERR_CUDA;
    }
    h->tmap_ptr[c][kind] = h->f[c];
    h->tmap_bn[c][kind] = BN;
    h->tmap_lanes[c][kind] = lanes;
  }
  *out = &h->tmap[c][kind];
  return FDTD_OK;
}

template <typename T>
size_t tma_smem_bytes(int lanes, int BN, int P, int nst) {
  return 2 * (size_t)nst * BN * lanes * sizeof(T) + 6 * (size_t)(P | 1) * lanes * sizeof(T) +
         (size_t)nst * sizeof(uint64_t);
}

// The TMA kernels take up to 227 KB of dynamic shared memory (set once per
// instantiation, outside any stream capture).
template <typename T, int LANES, int MINB, int NST>
cudaError_t ensure_tma_attr() {
  static bool attr_set = false;
  if (attr_set) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fdtd::proc_strided_tma_kernel<T, LANES, tma_L<T>(), MINB, NST>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fdtd::proc_strided_tma_st_kernel<T, LANES, tma_L<T>(), MINB, NST>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) attr_set = true;
  return e;
}

template <typename T, int LANES, int MINB, int NST>
int launch_strided_tma(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  constexpr int L = tma_L<T>();
  const int BN = ((g.N + 7) / 8) * 8;
  const int P = segments(g.N, L, LANES);
  const int kind = g.axis == AX_Y ? 0 : 1;
  const CUtensorMap *tE, *tH;
  int rc = get_tmap(h, g.ec, kind, BN, LANES, &tE);
  if (rc) return rc;
  if ((rc = get_tmap(h, g.hc, kind, BN, LANES, &tH))) return rc;
  fdtd::TmaTiles q;
  q.BN = BN;
  q.zbox = kind;
  q.tiles_x = (g.lane_hi + LANES - 1) / LANES;
  q.n_tiles = q.tiles_x * g.n_o;
  // outputs written from registers: with the three pairs of a procedure on
  // parallel branches the step is 1.8 % faster at 256^3 than with the
  // outputs staged in shared memory and written by TMA stores, although one
  // launch alone is 5 % slower; tune[1] bit 2: TMA stores
  const bool st = (h->desc.tune[1] & 4) != 0;
  const size_t smem = tma_smem_bytes<T>(LANES, BN, P, NST) + (st ? 2 * (size_t)BN * LANES * sizeof(T) : 0);
  auto kern = st ? fdtd::proc_strided_tma_st_kernel<T, LANES, L, MINB, NST>
                 : fdtd::proc_strided_tma_kernel<T, LANES, L, MINB, NST>;
  CK((ensure_tma_attr<T, LANES, MINB, NST>()));
  const int grid = std::min(q.n_tiles, MINB * h->num_sms);
  kern<<<grid, P * LANES, smem, h->stream>>>(*tE, *tH, p, q);
  return FDTD_OK;
}

// TMA-fed x lines (proc_rows_tma_kernel), on request (tune[1] bit 4): FP32
// fields, homogeneous media, 128 < N <= 256 (8 nodes per lane), R = 8
// consumer warps per block; bits 5-6 pick the ring depth and blocks per SM
// (0: 3 stages x 4 blocks, 1: 2 x 4, 2: 4 x 3, 3: 2 x 6).  Measured at 256^3
// per launch: 67.6 / 63.8 / 64.7 / 118 us against 58.9 us for the
// one-warp-per-line kernel, which stays the default: with the loads off the
// critical path the solve itself binds (instruction issue at 58 % with 32
// consumer warps per SM, against 66 % with 40 warps).
constexpr int kRowsR = 8;

bool rows_tma_eligible(const fdtd_t* h, const PairGeom& g) {
  return h->use_tma && h->prec == FDTD_F32 && !h->per_node && g.rows && (h->desc.tune[1] & 16) != 0 &&
         g.N > 128 && g.N <= 256 && rows_L(h, g) == 8 && tensor_map_encoder() != nullptr;
}

template <int NST, int MINB>
cudaError_t ensure_rows_tma_attr_one() {
  static bool set = false;
  if (set) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fdtd::proc_rows_tma_kernel<float, 8, kRowsR, NST, MINB, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fdtd::proc_rows_tma_kernel<float, 8, kRowsR, NST, MINB, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) set = true;
  return e;
}

// Set once per instantiation, outside any stream capture.
cudaError_t ensure_rows_tma_attr() {
  cudaError_t e = ensure_rows_tma_attr_one<3, 4>();
  if (e == cudaSuccess) e = ensure_rows_tma_attr_one<2, 4>();
  if (e == cudaSuccess) e = ensure_rows_tma_attr_one<4, 3>();
  if (e == cudaSuccess) e = ensure_rows_tma_attr_one<2, 6>();
  return e;
}

template <int NST, int MINB>
void launch_rows_tma_v(fdtd_t* h, const CUtensorMap* tE, const CUtensorMap* tH, const fdtd::PairParams<float>& p,
                       const fdtd::RowTiles& q) {
  const size_t smem = 2 * (size_t)NST * kRowsR * q.BN * sizeof(float) + 2 * (size_t)NST * sizeof(uint64_t);
  const int grid = std::min(q.n_tiles, MINB * h->num_sms);
  if (p.wall_fix)
    fdtd::proc_rows_tma_kernel<float, 8, kRowsR, NST, MINB, true><<<grid, (kRowsR + 1) * 32, smem, h->stream>>>(
        *tE, *tH, p, q);
  else
    fdtd::proc_rows_tma_kernel<float, 8, kRowsR, NST, MINB, false><<<grid, (kRowsR + 1) * 32, smem, h->stream>>>(
        *tE, *tH, p, q);
}

int launch_rows_tma(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<float>& p) {
  const int BN = ((g.N + 7) / 8) * 8;
  const CUtensorMap *tE, *tH;
  int rc = get_tmap(h, g.ec, 2, BN, kRowsR, &tE);
  if (rc) return rc;
  if ((rc = get_tmap(h, g.hc, 2, BN, kRowsR, &tH))) return rc;
  fdtd::RowTiles q;
  q.BN = BN;
  q.tpp = (g.n_o + kRowsR - 1) / kRowsR;
  q.n_tiles = q.tpp * g.n_o2;
  CK(ensure_rows_tma_attr());
  switch ((h->desc.tune[1] >> 5) & 3) {
    case 1: launch_rows_tma_v<2, 4>(h, tE, tH, p, q); break;
    case 2: launch_rows_tma_v<4, 3>(h, tE, tH, p, q); break;
    case 3: launch_rows_tma_v<2, 6>(h, tE, tH, p, q); break;
    default: launch_rows_tma_v<3, 4>(h, tE, tH, p, q); break;
  }
  return FDTD_OK;
}

int take_event(fdtd_t* h, int* idx) {
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  h->ev_pool.push_back(e);
  *idx = (int)h->ev_pool.size() - 1;
  return FDTD_OK;
}

int resolve_events(fdtd_t* h) {
  if (h->ev_rec.empty()) return FDTD_OK;
  CK(cudaStreamSynchronize(h->stream));
  for (auto& r : h->ev_rec) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, h->ev_pool[r.second.first], h->ev_pool[r.second.second]));
    h->timed_ms[r.first] += ms;
    h->timed_launches[r.first] += 1;
  }
  h->ev_rec.clear();
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  return FDTD_OK;
}

// General media (per-node mu): y/z lines 16 lanes x 8 nodes, x lines one
// warp per line (lines of at most 256 cells, checked by set_material).
template <typename T>
int launch_pair_gm(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  if (g.rows) {
    const int wpb = 8;
    const unsigned blocks = (unsigned)((g.n_lines() + wpb - 1) / wpb);
    switch (pick_rows_L(g.N)) {
      case 1: fdtd::proc_rows_gm_kernel<T, 1><<<blocks, wpb * 32, 0, h->stream>>>(p); break;
      case 2: fdtd::proc_rows_gm_kernel<T, 2><<<blocks, wpb * 32, 0, h->stream>>>(p); break;
      case 4: fdtd::proc_rows_gm_kernel<T, 4><<<blocks, wpb * 32, 0, h->stream>>>(p); break;
      case 8: fdtd::proc_rows_gm_kernel<T, 8><<<blocks, wpb * 32, 0, h->stream>>>(p); break;
      default: return FDTD_ERR_UNSUPPORTED;
    }
  } else {
    constexpr int LANES = 16, L = 8;
    const int P = segments(g.N, L, LANES);
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, fdtd::proc_strided_gm_kernel<T, LANES, L>));
    if (P > 32 || P * LANES > fa.maxThreadsPerBlock) return FDTD_ERR_UNSUPPORTED;
    dim3 grid((unsigned)((g.lane_hi + LANES - 1) / LANES), (unsigned)g.n_o);
    const size_t smem = 6 * (size_t)(P | 1) * LANES * sizeof(T);
    fdtd::proc_strided_gm_kernel<T, LANES, L><<<grid, P * LANES, smem, h->stream>>>(p);
  }
  CK(cudaGetLastError());
  return FDTD_OK;
}

// Fourth-order differences.  The procedure on lines of at most 512 cells
// runs the block-tiled kernel (chunks of 32 nodes: CH = 2, 8 or 16); longer
// lines, the explicit operator and tune[1] bit 9 take one thread per line
// (128 per block).  FP64 fields keep one thread per line: their work is
// bound by the FP64 pipe, which the tiled kernel's half-filled sweep warps
// (16 lines per block) use at half rate (measured at 256^3: 1.02 against
// 0.84 ms per launch on y and z lines; on x lines 0.99 against 1.40 ms alone,
// but a graph-replayed step of 6.5 against 4.7 ms with the three pairs
// running concurrently).

template <typename T>
size_t line4_tile_smem(const PairGeom& g) {
  return 2 * (size_t)g.N * fdtd::line4_tile_stride<T>(g.rows) * sizeof(T);
}

template <typename T, bool ROWS, int CH>
cudaError_t set_line4_tile_attr() {
  return cudaFuncSetAttribute(fdtd::proc_line4_tile_kernel<T, ROWS, CH>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * (size_t)32 * CH * fdtd::line4_tile_stride<T>(ROWS) * sizeof(T)));
}

// Dynamic shared memory limits of the tiled kernels (set outside any stream
// capture, from fdtd_set_order).
template <typename T>
cudaError_t ensure_line4_tile_attr() {
  static bool attr_set = false;
  if (attr_set) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  const cudaError_t r[6] = {set_line4_tile_attr<T, true, 2>(),   set_line4_tile_attr<T, true, 8>(),
                            set_line4_tile_attr<T, true, 16>(),  set_line4_tile_attr<T, false, 2>(),
                            set_line4_tile_attr<T, false, 8>(), set_line4_tile_attr<T, false, 16>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  if (e == cudaSuccess) attr_set = true;
  return e;
}

template <typename T>
bool line4_tile_eligible(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  if ((h->desc.tune[1] & 512) != 0 || g.N > kLine4TileMaxN || sizeof(T) != 4) return false;
  // the y/z tiles move 16-byte vectors
  for (const void* q : {(const void*)p.e_in, (const void*)p.h_in, (const void*)p.e_out, (const void*)p.h_out})
    if (((uintptr_t)q & 15) != 0) return false;
  return true;
}

template <typename T, bool ROWS, int CH>
void launch_line4_tile_ch(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  constexpr int LN = fdtd::line4_tile_lines<T>();
  const long long blocks = ROWS ? (g.n_lines() + LN - 1) / LN
                                : (long long)((g.lane_hi + LN - 1) / LN) * g.n_o;
  fdtd::proc_line4_tile_kernel<T, ROWS, CH><<<(unsigned)blocks, 256, line4_tile_smem<T>(g), h->stream>>>(p);
}

template <typename T, bool ROWS>
void launch_line4_tile(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  switch (fdtd::line4_tile_ch(g.N)) {
    case 2: launch_line4_tile_ch<T, ROWS, 2>(h, g, p); break;
    case 8: launch_line4_tile_ch<T, ROWS, 8>(h, g, p); break;
    default: launch_line4_tile_ch<T, ROWS, 16>(h, g, p); break;
  }
}

template <typename T>
void launch_line4_raw(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, int mode) {
  if (mode == 0 && line4_tile_eligible(h, g, p)) {
    if constexpr (sizeof(T) == 4) {
      if (g.rows) launch_line4_tile<T, true>(h, g, p);
      else launch_line4_tile<T, false>(h, g, p);
    }
    return;
  }
  const long long nl = g.n_lines();
  const unsigned blocks = (unsigned)std::min<long long>((nl + 127) / 128, 152LL * 64);
  fdtd::proc_line4_kernel<T><<<blocks, 128, 0, h->stream>>>(p, g.rows ? 1 : 0, mode);
}

template <typename T>
int launch_line4(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p, int mode) {
  if (!h->tmp4) return FDTD_ERR_STATE;
  h->launches++;
  launch_line4_raw<T>(h, g, p, mode);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// FP64 y/z lines (homogeneous media with the tables on every node, or
// per-node media with uniform mu), pairs of at least kSeqMinLines lines, take
// one thread per line (proc_strided_seq_kernel)
// once the scratch of its forward values exists (ensure_yseq, before the
// first step); tune[1] bit 10 keeps the segmented kernel.  Measured: 256^3
// (65,280 lines per pair) 8.5 G cell-steps/s against 7.4 G segmented; 128^3
// (16,256 lines, under one block per SM) 6.5 G against 7.8 G.
constexpr long long kSeqMinLines = 32768;
bool seq_wanted(const fdtd_t* h) {
  return h->prec == FDTD_F64 && !h->mu_var && h->order == 2 && (h->desc.tune[1] & 1024) == 0;
}

template <typename T>
bool seq_eligible(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  if (!seq_wanted(h) || !h->yseq || g.rows || p.nkd != nullptr || p.d_out != nullptr || g.N < 2 ||
      g.n_lines() < kSeqMinLines)
    return false;
  return p.nq != nullptr || (p.tab != nullptr && p.tables_only);
}

int ensure_yseq(fdtd_t* h) {
  if (!seq_wanted(h) || h->yseq) return FDTD_OK;
  CK(dev_malloc(&h->yseq, 3 * (size_t)h->count * h->esize));
  CK(cudaMemsetAsync(h->yseq, 0, 3 * (size_t)h->count * h->esize, h->stream));
  return FDTD_OK;
}

template <typename T>
int launch_pair(fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p) {
  if (g.empty()) return FDTD_OK;
  if (h->order == 4 && !h->tmp4) return FDTD_ERR_STATE;
  if (p.nkd) {
    h->launches++;
    return launch_pair_gm<T>(h, g, p);
  }
  const bool pn = h->per_node;
  const int cls = g.axis == AX_Y ? 0 : (g.axis == AX_Z ? 1 : 2);
  int ev0 = -1, ev1 = -1;
  if (h->timing) {
    int rc = take_event(h, &ev0);
    if (rc) return rc;
    if ((rc = take_event(h, &ev1))) return rc;
    CK(cudaEventRecord(h->ev_pool[ev0], h->stream));
  }
  h->launches++;
  if (h->order == 4) {
    launch_line4_raw<T>(h, g, p, 0);
  } else if (sizeof(T) == 8 && seq_eligible(h, g, p)) {
    if constexpr (sizeof(T) == 8) {
      const long long nl = g.n_lines();
      T* ys = (T*)h->yseq + (size_t)g.ec * h->count;
      const unsigned blocks = (unsigned)((nl + 127) / 128);
      if (p.nq) fdtd::proc_strided_seq_kernel<T, true><<<blocks, 128, 0, h->stream>>>(p, ys);
      else fdtd::proc_strided_seq_kernel<T, false><<<blocks, 128, 0, h->stream>>>(p, ys);
    }
  } else if (sizeof(T) == 8 && g.rows && rows_lanes(h, g) < 32) {
    if constexpr (sizeof(T) == 8) launch_rows_lpl<T>(h, g, p, rows_lanes(h, g));
  } else if (sizeof(T) == 4 && rows_tma_eligible(h, g) && p.e_in == (const T*)h->f[g.ec] &&
             p.h_in == (const T*)h->f[g.hc]) {
    // the tensor maps describe the state arrays; other inputs (scratch) take
    // the one-warp-per-line kernel
    if constexpr (sizeof(T) == 4) {
      if (int rc = launch_rows_tma(h, g, p)) return rc;
    }
  } else if (g.rows) {
    switch (pick_rows_L(g.N)) {
      case 1: launch_rows_L<T, 1>(h, g, p, pn); break;
      case 2: launch_rows_L<T, 2>(h, g, p, pn); break;
      case 4: launch_rows_L<T, 4>(h, g, p, pn); break;
      case 8: launch_rows_L<T, 8>(h, g, p, pn); break;
      case 12: launch_rows_L<T, 12>(h, g, p, pn); break;
      case 16: launch_rows_L<T, 16>(h, g, p, pn); break;
      case 24: launch_rows_L<T, 24>(h, g, p, pn); break;
      case 32: launch_rows_L<T, 32>(h, g, p, pn); break;
      default: return FDTD_ERR_UNSUPPORTED;
    }
  } else if (sizeof(T) == 4 && tma_eligible(h, g) && p.e_in == p.e_out && p.e_in == (const T*)h->f[g.ec] &&
             p.h_in == (const T*)h->f[g.hc]) {
    // 16-line tiles, two blocks per SM, two-stage ring (measured at 256^3:
    // a three-stage ring 9 % slower, three blocks per SM 12 % slower, 32-line
    // tiles with one block per SM equal)
    if constexpr (sizeof(T) == 4) {
      if (int rc = launch_strided_tma<T, 16, 2, 2>(h, g, p)) return rc;
    }
  } else {
    const StridedCfg& cfg = h->strided_cfg[g.axis == AX_Y ? 0 : 1];
    if (!cfg.ok) return FDTD_ERR_UNSUPPORTED;
    launch_strided<T>(h, g, p, pn, cfg.lanes, cfg.L);
  }
  CK(cudaGetLastError());
  if (h->timing) {
    CK(cudaEventRecord(h->ev_pool[ev1], h->stream));
    h->ev_rec.push_back({cls, {ev0, ev1}});
    // resolve in batches so the pool stays small
    if (h->ev_rec.size() >= 4096) {
      int rc = resolve_events(h);
      if (rc) return rc;
    }
  }
  return FDTD_OK;
}

// One updating procedure.  sgn = -1 runs the inverse procedure (length -h),
// whose tridiagonal matrices are the same and whose couplings flip sign.
template <typename T>
int run_procedure(fdtd_t* h, int slot, double sgn, double alpha, double beta, double kd_mul,
                  void* const* in, void* const* out) {
  const ProcCoef& P = h->proc[slot];
  NvtxScope range(P.op == 0 ? "procedure A" : "procedure B");
  for (int q = 0; q < 3; ++q) {
    const PairGeom& g = h->geom[P.op][q];
    fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], sgn, alpha, beta, kd_mul, in, out);
    int rc = launch_pair<T>(h, g, p);
    if (rc) return rc;
  }
  return FDTD_OK;
}

long long elem_index(const fdtd_t* h, int i, int j, int k) {
  return (long long)k * h->plane + (long long)j * h->pitch + i;
}

// value added to one sample of an array (a point source)
int add_point(fdtd_t* h, void* arr, double value) {
  if (value == 0.0 || h->src_comp < 0) return FDTD_OK;
  const long long at = elem_index(h, h->src_i, h->src_j, h->src_k);
  h->launches++;
  if (h->prec == FDTD_F64)
    fdtd::add_point_kernel<double><<<1, 32, 0, h->stream>>>((double*)arr, at, value);
  else
    fdtd::add_point_kernel<float><<<1, 32, 0, h->stream>>>((float*)arr, at, value);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// The forward procedure, in place: E <- w - E, H <- H + kd dw.  A point
// source enters as rhs_src added to the implicit right-hand side (applied by
// adding it to E before the solve and once more to the new E, since the new
// E subtracts the E the solve saw) and post_src added to the new E.
int procedure(fdtd_t* h, int slot, double rhs_src, double post_src) {
  int rc;
  if (h->src_comp >= 0 && rhs_src != 0.0) {
    if ((rc = add_point(h, h->f[h->src_comp], rhs_src))) return rc;
  }
  rc = h->prec == FDTD_F64 ? run_procedure<double>(h, slot, 1.0, 1.0, -1.0, 1.0, h->f, h->f)
                           : run_procedure<float>(h, slot, 1.0, 1.0, -1.0, 1.0, h->f, h->f);
  if (rc) return rc;
  if (h->src_comp >= 0 && (rhs_src != 0.0 || post_src != 0.0))
    return add_point(h, h->f[h->src_comp], rhs_src + post_src);
  return FDTD_OK;
}

int procedure_ex(fdtd_t* h, int slot, double sgn, double alpha, double beta, double kd_mul,
                 void* const* in, void* const* out) {
  return h->prec == FDTD_F64 ? run_procedure<double>(h, slot, sgn, alpha, beta, kd_mul, in, out)
                             : run_procedure<float>(h, slot, sgn, alpha, beta, kd_mul, in, out);
}

// The forward procedure with a right-hand-side source made of two terms
// (c fa + c fb), each added as its own rounded value before the solve and
// again to the new E: the FLOD2 B procedure, whose source is the mean of the
// samples on either side of t_{n+1}.  The graph path adds the same terms in
// the same order.
int procedure_two_terms(fdtd_t* h, int slot, double ta, double tb) {
  int rc;
  if ((rc = add_point(h, h->f[h->src_comp < 0 ? 0 : h->src_comp], ta))) return rc;
  if ((rc = add_point(h, h->f[h->src_comp < 0 ? 0 : h->src_comp], tb))) return rc;
  rc = procedure_ex(h, slot, 1.0, 1.0, -1.0, 1.0, h->f, h->f);
  if (rc) return rc;
  if ((rc = add_point(h, h->f[h->src_comp < 0 ? 0 : h->src_comp], ta))) return rc;
  return add_point(h, h->f[h->src_comp < 0 ? 0 : h->src_comp], tb);
}

int ensure_scratch(fdtd_t* h) {
  for (int c = 0; c < 6; ++c) {
    if (!h->scratch[c]) {
      CK(dev_malloc((void**)&h->scratch[c], (size_t)h->count * h->esize));
      CK(cudaMemsetAsync(h->scratch[c], 0, (size_t)h->count * h->esize, h->stream));
    }
  }
  return FDTD_OK;
}

int copy_state_to_scratch(fdtd_t* h) {
  int rc = ensure_scratch(h);
  if (rc) return rc;
  for (int c = 0; c < 6; ++c)
    CK(cudaMemcpyAsync(h->scratch[c], h->f[c], (size_t)h->count * h->esize, cudaMemcpyDeviceToDevice,
                       h->stream));
  return FDTD_OK;
}

double source_value(const fdtd_t* h, long long n) {
  // f_E at the source sample for step n: -I(t_n + dt/2)/(A eps)
  if (h->src_comp < 0 || n < 0 || n >= (long long)h->src_current.size()) return 0.0;
  return h->src_scale * h->src_current[(size_t)n];
}

int copy_uncovered_to_scratch(fdtd_t* h, int slot);

// FADI input initialization (Eq. 10 with Eqs. 7, 8a): v^0 = (I + dt/2 B) u^0
// plus the first sub-step's source (dt/2) f.
template <typename T>
int fadi_init_t(fdtd_t* h) {
  // the B pairs write their lines of all six arrays into scratch; what no
  // line covers keeps its value: the H samples on the walls (normal H, not
  // updated) and the arrays of a pair without unknowns are copied, while E
  // outside the lines is the walls and the row padding, zero in every array
  int rc = copy_uncovered_to_scratch(h, 1);
  if (rc) return rc;
  const ProcCoef& P = h->proc[1];
  for (int q = 0; q < 3; ++q) {
    const PairGeom& g = h->geom[1][q];
    if (g.empty()) continue;
    // (I + tau B) with tau = dt/2: kb = s*b/d_eta with b = dt/(2 eps) = tau/eps
    fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], 1.0, 1.0, 0.0, 1.0, h->f, h->scratch);
    if (h->order == 4) {
      if (int rc4 = launch_line4<T>(h, g, p, 1)) return rc4;
      continue;
    }
    const long long total = g.n_lines() * g.N;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 32);
    h->launches++;
    if (h->per_node)
      fdtd::explicit_pair_kernel<T, true><<<blocks, 256, 0, h->stream>>>(p, g.rows ? 1 : 0);
    else
      fdtd::explicit_pair_kernel<T, false><<<blocks, 256, 0, h->stream>>>(p, g.rows ? 1 : 0);
    CK(cudaGetLastError());
  }
  if (h->lossy) {
    // the loss part of (I + dt/2 B): E -= (dt/2)(sigma/(2 eps)) E of u^0
    for (int c = 0; c < 3; ++c) {
      h->launches++;
      fdtd::loss_scale_kernel<T><<<152 * 8, 256, 0, h->stream>>>(
          (T*)h->scratch[c], (const T*)h->f[c], h->sig_node[c], h->per_node ? h->eps_node[c] : nullptr, h->sigma_u,
          h->per_node ? 1.0 : h->eps_r, 0.25 * h->dt / kEps0, h->count);
      CK(cudaGetLastError());
    }
  }
  for (int c = 0; c < 6; ++c) std::swap(h->f[c], h->scratch[c]);
  const double f0 = source_value(h, h->steps);
  if (f0 != 0.0) {
    h->launches++;
    fdtd::add_point_kernel<T><<<1, 32, 0, h->stream>>>(
        (T*)h->f[h->src_comp], elem_index(h, h->src_i, h->src_j, h->src_k), 0.5 * h->dt * f0);
    CK(cudaGetLastError());
  }
  h->output_valid = false;
  return FDTD_OK;
}

int scheme_init(fdtd_t* h) {
  if (!h->pending_init) return FDTD_OK;
  int rc = FDTD_OK;
  if (h->scheme == FDTD_FADI) {
    rc = h->prec == FDTD_F64 ? fadi_init_t<double>(h) : fadi_init_t<float>(h);
  } else if (h->scheme == FDTD_FLOD2) {
    // Eq. 22: (1/2 I - dt/8 B) v = u^n + (dt/8) f(t_n + dt/2), u^{n+1/4} = v - u^n
    // (procedure of length dt/2; n = the steps taken so far)
    rc = procedure(h, 2, 0.125 * h->dt * source_value(h, h->steps), 0.0);
  }
  if (rc) return rc;
  h->pending_init = false;
  return FDTD_OK;
}

template <typename T>
int record_probes(fdtd_t* h, int mode, double post, void* const* arrays) {
  if (h->nprobes == 0) return FDTD_OK;
  fdtd::ProbeParams<T> pp;
  pp.n = h->nprobes;
  const long long src_at = h->src_comp >= 0 ? elem_index(h, h->src_i, h->src_j, h->src_k) : -1;
  for (int q = 0; q < h->nprobes; ++q) {
    pp.arr[q] = (const T*)arrays[h->probe_comp[q]];
    pp.at[q] = h->probe_at[q];
    pp.sub[q] = (h->probe_comp[q] == h->src_comp && h->probe_at[q] == src_at) ? post : 0.0;
  }
  h->launches++;
  fdtd::probe_kernel<T><<<1, 32, 0, h->stream>>>(pp, h->d_stash, h->d_probe, h->probe_cap, h->steps, mode);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// mode 1 (FADI, after B): post = the source just added after the B
// subtraction, which the output w_B/2 does not contain
int probes(fdtd_t* h, int mode, double post = 0.0, void* const* arrays = nullptr) {
  if (!arrays) arrays = h->f;
  return h->prec == FDTD_F64 ? record_probes<double>(h, mode, post, arrays)
                             : record_probes<float>(h, mode, post, arrays);
}

int ensure_probe_capacity(fdtd_t* h, long long need) {
  if (h->nprobes == 0 || need <= h->probe_cap) return FDTD_OK;
  long long cap = std::max<long long>(need, 2 * h->probe_cap);
  cap = std::max<long long>(cap, 1024);
  double* np = nullptr;
  CK(dev_malloc((void**)&np, sizeof(double) * fdtd::kMaxProbes * cap));
  CK(cudaMemsetAsync(np, 0, sizeof(double) * fdtd::kMaxProbes * cap, h->stream));
  if (h->d_probe) {
    CK(cudaMemcpy2DAsync(np, sizeof(double) * cap, h->d_probe, sizeof(double) * h->probe_cap,
                         sizeof(double) * h->probe_cap, fdtd::kMaxProbes, cudaMemcpyDeviceToDevice,
                         h->stream));
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(h->d_probe);
  }
  h->d_probe = np;
  h->probe_cap = cap;
  return FDTD_OK;
}

// One time step of the handle's scheme (Sec. II):
//   FADI  P_A(dt), P_B(dt) on the auxiliary state, the source (dt/2) f added
//         to the state after each procedure (it is part of v, Eqs. 2, 8);
//   FLOD  P_A(dt), P_B(dt) with +(dt/4) f in each implicit RHS (Eq. 15);
//   FSS   P_A(dt/2), P_B(dt), P_A(dt/2) with +(h/4) f (Eq. 17);
//   FLOD2 FLOD main iterations (Eq. 21).
int physical_to_scratch(fdtd_t* h, long long n_next = -1);

// Drop the captured step.  Replays still in flight on the (non-blocking)
// replay stream finish first: callers go on to rewrite or free buffers the
// graph reads (source table, coefficients).
void graph_release(fdtd_t* h) {
  if (h->g_run) cudaStreamSynchronize(h->g_run);
  if (h->g_exec) cudaGraphExecDestroy(h->g_exec);
  h->g_exec = nullptr;
  h->g_bound.clear();
}

bool graph_usable(const fdtd_t* h) {
  return !h->timing && h->nprobes == 0 && (h->desc.tune[1] & 8) == 0 &&
         (h->src_comp < 0 || h->d_srcval != nullptr);
}

// nsteps steps as replays of a captured one-step graph: each procedure forks
// its three pair launches (disjoint arrays) onto parallel branches and joins
// them before the next procedure; a point source is added by kernels that
// read each step's value from a device table indexed by a device step
// counter.  Same kernels, same arguments, same results as one_step.
int ensure_branches(fdtd_t* h);

int step_graph(fdtd_t* h, int64_t nsteps) {
  if (int rc = ensure_branches(h)) return rc;
  const bool src = h->src_comp >= 0;
  std::vector<const void*> ptrs(h->f, h->f + 6);
  if (!h->g_exec || ptrs != h->g_bound) {
    graph_release(h);
    if (h->prec == FDTD_F32) CK((ensure_tma_attr<float, 16, 2, 2>()));
    if (h->prec == FDTD_F32) CK(ensure_rows_tma_attr());
    static const int seq_fss[3] = {0, 1, 0};
    static const int seq_two[2] = {0, 1};
    const int* seq = h->scheme == FDTD_FSS ? seq_fss : seq_two;
    const int nproc = h->scheme == FDTD_FSS ? 3 : 2;
    // the source terms of one_step: coefficient of f added before and after
    // each procedure (0 = none), and the step offset of the value after it
    const double dt = h->dt;
    double pre[3] = {0, 0, 0}, post[3] = {0, 0, 0};
    double pre2[3] = {0, 0, 0}, post2[3] = {0, 0, 0};   // second terms, step offset 1
    int post_off[3] = {0, 0, 0};
    if (h->scheme == FDTD_FADI) {
      post[0] = 0.5 * dt;
      post[1] = 0.5 * dt;
      post_off[1] = 1;
    } else if (h->scheme == FDTD_FSS) {
      pre[0] = post[0] = 0.125 * dt;
      pre[1] = post[1] = 0.25 * dt;
      pre[2] = post[2] = 0.125 * dt;
    } else if (h->scheme == FDTD_FLOD2) {
      // B: (dt/4) of the mean of f(t_n + dt/2) and f(t_n + 3dt/2), as two
      // terms (dt/8) f of offsets 0 and 1 (procedure_two_terms)
      pre[0] = post[0] = 0.25 * dt;
      pre[1] = post[1] = 0.125 * dt;
      pre2[1] = post2[1] = 0.125 * dt;
    } else {
      pre[0] = post[0] = 0.25 * dt;
      pre[1] = post[1] = 0.25 * dt;
    }
    if (src && !h->d_step) CK(dev_malloc((void**)&h->d_step, sizeof(long long)));
    const long long src_at = src ? elem_index(h, h->src_i, h->src_j, h->src_k) : 0;
    auto add_src = [&](double coef, int off) -> cudaError_t {
      if (!src || coef == 0.0) return cudaSuccess;
      if (h->prec == FDTD_F64)
        fdtd::add_point_table_kernel<double><<<1, 32, 0, h->g_run>>>((double*)h->f[h->src_comp], src_at,
                                                                     h->d_srcval, h->srcval_len, h->d_step, off, coef);
      else
        fdtd::add_point_table_kernel<float><<<1, 32, 0, h->g_run>>>((float*)h->f[h->src_comp], src_at, h->d_srcval,
                                                                    h->srcval_len, h->d_step, off, coef);
      h->launches++;
      return cudaGetLastError();
    };
    cudaStream_t home = h->stream;
    const long long before = h->launches;
    NvtxScope range("step graph capture");
    CK(cudaStreamBeginCapture(h->g_run, cudaStreamCaptureModeThreadLocal));
    int rc = FDTD_OK;
    for (int k = 0; k < nproc && rc == FDTD_OK; ++k) {
      if (add_src(pre[k], 0) != cudaSuccess) rc = FDTD_ERR_CUDA;
      if (rc == FDTD_OK && add_src(pre2[k], 1) != cudaSuccess) rc = FDTD_ERR_CUDA;
      if (rc == FDTD_OK && cudaEventRecord(h->g_fork, h->g_run) != cudaSuccess) rc = FDTD_ERR_CUDA;
      const ProcCoef& P = h->proc[seq[k]];
      for (int q = 0; q < 3 && rc == FDTD_OK; ++q) {
        if (cudaStreamWaitEvent(h->g_br[q], h->g_fork, 0) != cudaSuccess) { rc = FDTD_ERR_CUDA; break; }
        h->stream = h->g_br[q];
        const PairGeom& g = h->geom[P.op][q];
        if (h->prec == FDTD_F64) {
          fdtd::PairParams<double> p = make_params<double>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, h->f, h->f);
          rc = launch_pair<double>(h, g, p);
        } else {
          fdtd::PairParams<float> p = make_params<float>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, h->f, h->f);
          rc = launch_pair<float>(h, g, p);
        }
        h->stream = home;
        if (rc == FDTD_OK && (cudaEventRecord(h->g_join[q], h->g_br[q]) != cudaSuccess ||
                              cudaStreamWaitEvent(h->g_run, h->g_join[q], 0) != cudaSuccess))
          rc = FDTD_ERR_CUDA;
      }
      if (rc == FDTD_OK && add_src(post[k], post_off[k]) != cudaSuccess) rc = FDTD_ERR_CUDA;
      if (rc == FDTD_OK && add_src(post2[k], 1) != cudaSuccess) rc = FDTD_ERR_CUDA;
    }
    if (rc == FDTD_OK && src) {
      fdtd::step_counter_kernel<<<1, 32, 0, h->g_run>>>(h->d_step, 0, 1);
      h->launches++;
      if (cudaGetLastError() != cudaSuccess) rc = FDTD_ERR_CUDA;
    }
    h->stream = home;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->g_run, &graph);
    h->g_kernels = h->launches - before;
    h->launches = before;
    if (rc != FDTD_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != FDTD_OK ? rc : cuda_fail(h, e);
    }
    const cudaError_t ie = cudaGraphInstantiate(&h->g_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ie);
    h->g_bound = ptrs;
  }
  CK(cudaEventRecord(h->g_in, h->stream));
  CK(cudaStreamWaitEvent(h->g_run, h->g_in, 0));
  if (src) {
    fdtd::step_counter_kernel<<<1, 32, 0, h->g_run>>>(h->d_step, h->steps, 0);
    CK(cudaGetLastError());
  }
  {
    NvtxScope range("step graph replays");
    for (int64_t k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(h->g_exec, h->g_run));
  }
  CK(cudaEventRecord(h->g_out, h->g_run));
  CK(cudaStreamWaitEvent(h->stream, h->g_out, 0));
  h->launches += nsteps * h->g_kernels;
  h->steps += nsteps;
  return FDTD_OK;
}

// The three pairs of one procedure touch disjoint arrays: launch(q) for
// q = 0..2 on three branch streams forked from and joined back into the
// handle's stream (launches inside launch() go to h->stream, which points
// at the branch meanwhile).
int ensure_branches(fdtd_t* h) {
  if (h->g_run) return FDTD_OK;
  CK(cudaStreamCreateWithFlags(&h->g_run, cudaStreamNonBlocking));
  for (int b = 0; b < 3; ++b) {
    CK(cudaStreamCreateWithFlags(&h->g_br[b], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->g_join[b], cudaEventDisableTiming));
  }
  CK(cudaEventCreateWithFlags(&h->g_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->g_out, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->g_fork, cudaEventDisableTiming));
  return FDTD_OK;
}

template <typename F>
int fork_pairs(fdtd_t* h, F&& launch) {
  int rc = ensure_branches(h);
  if (rc) return rc;
  cudaStream_t home = h->stream;
  CK(cudaEventRecord(h->g_fork, home));
  for (int q = 0; q < 3 && rc == FDTD_OK; ++q) {
    CK(cudaStreamWaitEvent(h->g_br[q], h->g_fork, 0));
    h->stream = h->g_br[q];
    rc = launch(q);
    h->stream = home;
    CK(cudaEventRecord(h->g_join[q], h->g_br[q]));
    CK(cudaStreamWaitEvent(home, h->g_join[q], 0));
  }
  h->stream = home;
  return rc;
}

int one_step(fdtd_t* h) {
  const long long n = h->steps;
  const double dt = h->dt;
  const double f = source_value(h, n);
  int rc;
  switch (h->scheme) {
    case FDTD_FADI: {
      const double fn = source_value(h, n + 1);
      if ((rc = procedure(h, 0, 0.0, 0.5 * dt * f))) return rc;
      if ((rc = probes(h, 0))) return rc;
      if ((rc = procedure(h, 1, 0.0, 0.5 * dt * fn))) return rc;
      if ((rc = probes(h, 1, 0.5 * dt * fn))) return rc;
      break;
    }
    case FDTD_FLOD:
    case FDTD_FLOD2: {
      if ((rc = procedure(h, 0, 0.25 * dt * f, 0.0))) return rc;
      if (h->scheme == FDTD_FLOD) {
        if ((rc = procedure(h, 1, 0.25 * dt * f, 0.0))) return rc;
      } else {
        // FLOD2's B procedure is centred on t_{n+1}: (dt/4) of the mean of
        // the samples at t_n + dt/2 and t_n + 3dt/2
        const double fn = source_value(h, n + 1);
        if ((rc = procedure_two_terms(h, 1, 0.125 * dt * f, 0.125 * dt * fn))) return rc;
      }
      if (h->nprobes) {
        if (h->scheme == FDTD_FLOD) {
          if ((rc = probes(h, 2))) return rc;
        } else {
          // probes of the FLOD2 physical field: output processing (Eq. 23)
          // of the new state into scratch, sampled there
          h->output_valid = false;
          if ((rc = physical_to_scratch(h, n + 1))) return rc;
          if ((rc = probes(h, 2, 0.0, h->scratch))) return rc;
        }
      }
      break;
    }
    case FDTD_FSS: {
      if ((rc = procedure(h, 0, 0.125 * dt * f, 0.0))) return rc;
      if ((rc = procedure(h, 1, 0.25 * dt * f, 0.0))) return rc;
      if ((rc = procedure(h, 0, 0.125 * dt * f, 0.0))) return rc;
      if ((rc = probes(h, 2))) return rc;
      break;
    }
    default:
      return FDTD_ERR_STATE;
  }
  h->steps++;
  return FDTD_OK;
}

// Scratch receives the B procedure's (or explicit operator's) output line by
// line; the samples no line of it covers keep the state's values: the three
// H components are copied whole (their samples on the walls, normal H, are
// in no line), and both arrays of a pair without unknowns (lines of one
// cell).  E outside the lines is the walls and the row padding, zero in the
// state and in scratch alike (no kernel writes a nonzero value there).
int copy_uncovered_to_scratch(fdtd_t* h, int slot) {
  int rc = ensure_scratch(h);
  if (rc) return rc;
  const ProcCoef& P = h->proc[slot];
  bool copied[6] = {false, false, false, false, false, false};
  for (int c = 3; c < 6; ++c) copied[c] = true;
  for (int q = 0; q < 3; ++q)
    if (h->geom[P.op][q].empty()) copied[h->geom[P.op][q].ec] = true;
  for (int c = 0; c < 6; ++c)
    if (copied[c])
      CK(cudaMemcpyAsync(h->scratch[c], h->f[c], (size_t)h->count * h->esize, cudaMemcpyDeviceToDevice,
                         h->stream));
  return FDTD_OK;
}

// Physical field into scratch (FADI: (I + dt/2 B)^{-1}(v - pending source),
// from Eqs. 2a, 8a, 9; FLOD2: output processing Eq. 23).  n_next: index of
// the step that would come next (-1: the steps taken so far).
int physical_to_scratch(fdtd_t* h, long long n_next) {
  if (n_next < 0) n_next = h->steps;
  if (h->output_valid) return FDTD_OK;
  int rc;
  if (h->pending_init || (h->scheme != FDTD_FADI && h->scheme != FDTD_FLOD2)) {
    if ((rc = copy_state_to_scratch(h))) return rc;
    h->output_valid = true;
    return FDTD_OK;
  }
  // The B pairs read the state and write scratch (out of place); what no
  // line covers is copied (copy_uncovered_to_scratch).  The source sample's
  // E component is copied to scratch first and adjusted there.
  const bool fadi = h->scheme == FDTD_FADI;
  const int slot = fadi ? (h->lossy ? 3 : 1) : (h->lossy ? 4 : 2);
  if ((rc = copy_uncovered_to_scratch(h, slot))) return rc;
  void* in[6];
  for (int c = 0; c < 6; ++c) in[c] = h->f[c];
  // FADI: u = (I + dt/2 B)^{-1} (v - (dt/2) f_pending), from Eqs. 2a, 8a and
  // 9: the B pairs' line systems with the couplings of a procedure of length
  // -dt; E_out = w/2 and H_out = H + (1/2) kd' dw.
  // FLOD2, Eq. 23: (1/2 I + dt/8 B) v = u^{n+5/4} - (dt/8) f(t_{n+1} + dt/2),
  // u^{n+1} = v - u^{n+5/4}; the source term is added before the solve and
  // once more to the new E (which subtracts the E the solve saw).
  const double adj = fadi ? -0.5 * h->dt * source_value(h, n_next) : -0.125 * h->dt * source_value(h, n_next);
  const bool src = h->src_comp >= 0 && adj != 0.0;
  if (src) {
    CK(cudaMemcpyAsync(h->scratch[h->src_comp], h->f[h->src_comp], (size_t)h->count * h->esize,
                       cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = add_point(h, h->scratch[h->src_comp], adj))) return rc;
    in[h->src_comp] = h->scratch[h->src_comp];
  }
  if (fadi) rc = procedure_ex(h, slot, -1.0, 0.5, 0.0, 0.5, in, h->scratch);
  else rc = procedure_ex(h, slot, -1.0, 1.0, -1.0, 1.0, in, h->scratch);
  if (rc) return rc;
  if (!fadi && src && (rc = add_point(h, h->scratch[h->src_comp], adj))) return rc;
  h->output_valid = true;
  return FDTD_OK;
}

int check_comp(int c) { return (c >= 0 && c < 6) ? FDTD_OK : FDTD_ERR_INVALID_ARG; }

// Did a kernel's bounded wait give up?  (Synchronises the stream.)
int check_device_flag(fdtd_t* h) {
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
#ifdef FDTD_BOUNDS
  int b = 0;
  CK(cudaMemcpyFromSymbol(&b, fdtd::g_bounds_err, sizeof(int)));
  if (b) return FDTD_ERR_BOUNDS;
#endif
  return v ? FDTD_ERR_TIMEOUT : FDTD_OK;
}

// f_E = -I / (A eps) at the source sample (A = the sample's dual-face area).
int refresh_src_scale(fdtd_t* h) {
  if (h->src_comp < 0) {
    h->src_scale = 0;
    return FDTD_OK;
  }
  double er = h->eps_r;
  if (h->per_node)
    CK(cudaMemcpy(&er, h->eps_node[h->src_comp] + elem_index(h, h->src_i, h->src_j, h->src_k), sizeof(double),
                  cudaMemcpyDeviceToHost));
  const double area = h->src_comp == EX ? h->dy * h->dz : (h->src_comp == EY ? h->dx * h->dz : h->dx * h->dy);
  h->src_scale = -1.0 / (area * kEps0 * er);
  // device copy of the per-step values for graph-replayed steps
  graph_release(h);
  const long long len = (long long)h->src_current.size();
  if (len != h->srcval_len) {
    if (h->d_srcval) cudaFree(h->d_srcval);
    h->d_srcval = nullptr;
    h->srcval_len = 0;
    CK(dev_malloc((void**)&h->d_srcval, sizeof(double) * (size_t)std::max(len, 1LL)));
    h->srcval_len = len;
  }
  std::vector<double> v((size_t)len);
  for (long long n = 0; n < len; ++n) v[(size_t)n] = source_value(h, n);
  if (len) CK(cudaMemcpy(h->d_srcval, v.data(), sizeof(double) * (size_t)len, cudaMemcpyHostToDevice));
  return FDTD_OK;
}

// Host copies go through a contiguous device staging buffer (one transfer
// at full link bandwidth, then a (un)pack kernel) instead of a row-by-row
// pitched copy; device-to-device copies stay pitched.
int ensure_stage(fdtd_t* h) {
  if (h->stage) return FDTD_OK;
  const size_t n = (size_t)(h->nx + 1) * (h->ny + 1) * (h->nz + 1);
  CK(dev_malloc((void**)&h->stage, n * h->esize));
  return FDTD_OK;
}

int stage_unpack(fdtd_t* h, int sx, int sy, int sz, void* dst_padded, const void* src = nullptr) {
  if (!src) src = h->stage;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((long long)sy * sz, 152LL * 16));
  if (h->prec == FDTD_F64)
    fdtd::unpack_kernel<double><<<blocks, 256, 0, h->stream>>>((const double*)src, (double*)dst_padded, sx, sy,
                                                               sz, h->pitch, h->plane);
  else
    fdtd::unpack_kernel<float><<<blocks, 256, 0, h->stream>>>((const float*)src, (float*)dst_padded, sx, sy, sz,
                                                              h->pitch, h->plane);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// The device address of page-locked (pinned) host memory, or nullptr for
// pageable memory (or when tune[1] bit 8 asks for the staged copies).  A
// kernel reads pinned memory in place over the host link as fast as a copy
// engine transfers it on this machine (about 210 GB/s, measured), without
// the staging buffer and its extra pass over device memory.
void* pinned_device_view(const fdtd_t* h, const void* host) {
  if (h->desc.tune[1] & 256) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int stage_pack(fdtd_t* h, int sx, int sy, int sz, const void* src_padded) {
  void* dst = h->stage;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((long long)sy * sz, 152LL * 16));
  if (h->prec == FDTD_F64)
    fdtd::pack_kernel<double><<<blocks, 256, 0, h->stream>>>((const double*)src_padded, (double*)dst, sx, sy, sz,
                                                             h->pitch, h->plane);
  else
    fdtd::pack_kernel<float><<<blocks, 256, 0, h->stream>>>((const float*)src_padded, (float*)dst, sx, sy, sz,
                                                            h->pitch, h->plane);
  CK(cudaGetLastError());
  return FDTD_OK;
}

int copy_component(fdtd_t* h, int comp, const void* src_padded, void* dst, int on_device) {
  int sx, sy, sz;
  comp_extent(comp, h->nx, h->ny, h->nz, &sx, &sy, &sz);
  if (!on_device) {
    // (packing straight into pinned host memory measured slower than the
    // staged pack and copy: 3.3 against 3.1 ms for the six 256^3 fields)
    int rc;
    if ((rc = ensure_stage(h))) return rc;
    if ((rc = stage_pack(h, sx, sy, sz, src_padded))) return rc;
    CK(cudaMemcpyAsync(dst, h->stage, (size_t)sx * sy * sz * h->esize, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
  }
  cudaMemcpy3DParms m = {};
  m.srcPtr = make_cudaPitchedPtr((void*)src_padded, (size_t)h->pitch * h->esize, (size_t)h->pitch,
                                 (size_t)(h->ny + 1));
  m.dstPtr = make_cudaPitchedPtr(dst, (size_t)sx * h->esize, (size_t)sx, (size_t)sy);
  m.extent = make_cudaExtent((size_t)sx * h->esize, (size_t)sy, (size_t)sz);
  m.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpy3DAsync(&m, h->stream));
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  return FDTD_OK;
}

int copy_in_component(fdtd_t* h, int comp, const void* src, void* dst_padded, int on_device) {
  int sx, sy, sz;
  comp_extent(comp, h->nx, h->ny, h->nz, &sx, &sy, &sz);
  if (!on_device) {
    int rc;
    if (const void* view = pinned_device_view(h, src)) {
      // pinned source: unpacked straight from it
      if ((rc = stage_unpack(h, sx, sy, sz, dst_padded, view))) return rc;
      CK(cudaStreamSynchronize(h->stream));
      return FDTD_OK;
    }
    if ((rc = ensure_stage(h))) return rc;
    CK(cudaMemcpyAsync(h->stage, src, (size_t)sx * sy * sz * h->esize, cudaMemcpyHostToDevice, h->stream));
    if ((rc = stage_unpack(h, sx, sy, sz, dst_padded))) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return FDTD_OK;
  }
  cudaMemcpy3DParms m = {};
  m.srcPtr = make_cudaPitchedPtr((void*)src, (size_t)sx * h->esize, (size_t)sx, (size_t)sy);
  m.dstPtr = make_cudaPitchedPtr(dst_padded, (size_t)h->pitch * h->esize, (size_t)h->pitch,
                                 (size_t)(h->ny + 1));
  m.extent = make_cudaExtent((size_t)sx * h->esize, (size_t)sy, (size_t)sz);
  m.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpy3DAsync(&m, h->stream));
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  return FDTD_OK;
}


int zero_walls(fdtd_t* h, int comp, void* arr) {
  if (comp >= 3) return FDTD_OK;
  h->launches++;
  if (h->prec == FDTD_F64)
    fdtd::zero_walls_kernel<double><<<1216, 256, 0, h->stream>>>((double*)arr, comp, h->nx, h->ny, h->nz, h->pitch,
                                                                 h->plane);
  else
    fdtd::zero_walls_kernel<float><<<1216, 256, 0, h->stream>>>((float*)arr, comp, h->nx, h->ny, h->nz, h->pitch,
                                                                h->plane);
  CK(cudaGetLastError());
  return FDTD_OK;
}

constexpr int kEnergyBlocks = 152 * 8;

// Per-block partial sums of the energy of the six arrays into
// partial[blocks], one launch (asynchronous on the handle's stream).
template <typename T>
int energy_launch(fdtd_t* h, void* const* arr, double* partial) {
  fdtd::Energy6 a;
  for (int c = 0; c < 6; ++c) {
    a.x[c] = arr[c];
    a.w[c] = c < 3 ? kEps0 * (h->per_node ? 1.0 : h->eps_r) : kMu0 * h->mu_r;
    a.wv[c] = c < 3 ? (h->per_node ? h->eps_node[c] : nullptr) : (h->mu_var ? h->mu_node[c - 3] : nullptr);
  }
  h->launches++;
  fdtd::weighted_sumsq6_kernel<T><<<kEnergyBlocks, 256, 0, h->stream>>>(a, h->count, partial);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// Read back and add up the partials (synchronises the stream).
int energy_sum(fdtd_t* h, const double* partial, double* out) {
  std::vector<double> part((size_t)kEnergyBlocks);
  CK(cudaMemcpyAsync(part.data(), partial, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  double s = 0;
  for (double v : part) s += v;
  *out = 0.5 * h->dx * h->dy * h->dz * s;
  return FDTD_OK;
}

int energy(fdtd_t* h, void* const* arr, double* out) {
  if (!h->d_partial) {
    CK(dev_malloc((void**)&h->d_partial, sizeof(double) * kEnergyBlocks));
    h->partial_n = kEnergyBlocks;
  }
  int rc = h->prec == FDTD_F64 ? energy_launch<double>(h, arr, h->d_partial)
                               : energy_launch<float>(h, arr, h->d_partial);
  if (rc) return rc;
  return energy_sum(h, h->d_partial, out);
}

// Reference of the scheme invariant for the growth check of fdtd_energy:
// after a change of fields, source or media, the invariant of the state as
// the next step starts from it, reduced on the device (read back only when
// fdtd_energy needs it).  A run with a source has no reference: its
// invariant changes legitimately.
int take_invariant_ref(fdtd_t* h) {
  if (!h->inv_dirty) return FDTD_OK;
  h->inv_dirty = false;
  h->inv_have = false;
  h->inv_ref = -1.0;
  if (h->src_comp >= 0) return FDTD_OK;
  if (!h->d_ref_partial) CK(dev_malloc((void**)&h->d_ref_partial, sizeof(double) * kEnergyBlocks));
  int rc = h->prec == FDTD_F64 ? energy_launch<double>(h, h->f, h->d_ref_partial)
                               : energy_launch<float>(h, h->f, h->d_ref_partial);
  if (rc) return rc;
  h->inv_have = true;
  return FDTD_OK;
}

// Relative growth of the invariant past its reference that fdtd_energy
// reports as FDTD_ERR_UNSTABLE.  Every procedure conserves it exactly in
// exact arithmetic; measured roundoff drift is about 1e-13 (FP64) and 1e-5
// (FP32) per thousand steps.
double invariant_growth_limit(const fdtd_t* h) { return h->prec == FDTD_F64 ? 1e-8 : 1e-2; }

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

int fdtd_debug_fail_alloc(int64_t n) {
  g_fail_alloc_in.store(n < 0 ? -1 : (long long)n);
  return FDTD_OK;
}

int fdtd_selftest_bounded_wait(int64_t limit_ns, int arrive, void* stream) {
  if (limit_ns <= 0 || limit_ns > 10000000000LL) return FDTD_ERR_INVALID_ARG;
  int* d_flag = nullptr;
  if (dev_malloc((void**)&d_flag, sizeof(int)) != cudaSuccess) return FDTD_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  int v = -1;
  fdtd::bounded_wait_probe_kernel<<<1, 32, 0, st>>>(d_flag, (unsigned long long)limit_ns, arrive ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_flag);
  if (e != cudaSuccess) {
    fprintf(stderr, "fdtd: CUDA error: %s\n", cudaGetErrorString(e));
    return FDTD_ERR_CUDA;
  }
  return v == 0 ? FDTD_OK : FDTD_ERR_TIMEOUT;
}

int fdtd_probe_fp64_fma(int64_t iters, double* flops_per_s, void* stream) {
  if (iters < 1 || iters > 1000000LL || !flops_per_s) return FDTD_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* d_out = nullptr;
  if (e == cudaSuccess && dev_malloc((void**)&d_out, sizeof(double)) != cudaSuccess) return FDTD_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  // 8 blocks of 256 threads per SM (64 warps), 8 independent chains each
  const int blocks = 8 * sms, threads = 256;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fdtd::fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(d_out, iters / 8 + 1, 0.999999, 1e-6, -1.0);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    fdtd::fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(d_out, iters, 0.999999, 1e-6, -1.0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess || ms <= 0.f) {
    fprintf(stderr, "fdtd: CUDA error: %s\n", cudaGetErrorString(e));
    return FDTD_ERR_CUDA;
  }
  *flops_per_s = 2.0 * 8.0 * (double)iters * (double)blocks * threads / (ms * 1e-3);
  return FDTD_OK;
}

const char* fdtd_strerror(int code) {
  switch (code) {
    case FDTD_OK: return "ok";
    case FDTD_ERR_INVALID_ARG: return "invalid argument";
    case FDTD_ERR_OOM: return "out of memory";
    case FDTD_ERR_CUDA: return "CUDA error (handle poisoned)";
    case FDTD_ERR_TIMEOUT: return "device wait timed out";
    case FDTD_ERR_UNSTABLE: return "non-finite field or invariant";
    case FDTD_ERR_UNSUPPORTED: return "unsupported in this build";
    case FDTD_ERR_STATE: return "call not valid in the handle's state";
    case FDTD_ERR_BOUNDS: return "a kernel index fell outside its array (bounds-checked build)";
    default: return "unknown error";
  }
}

int fdtd_create(const fdtd_desc* desc, void* stream, fdtd_t** out) {
  if (!desc || !out) return FDTD_ERR_INVALID_ARG;
  *out = nullptr;
  const fdtd_desc& d = *desc;
  if (d.nx < 2 || d.ny < 2 || d.nz < 1 || d.nx > 1024 || d.ny > 4096 || d.nz > 4096) return FDTD_ERR_INVALID_ARG;
  if (!(d.dx > 0) || !(d.dy > 0) || !(d.dz > 0) || !std::isfinite(d.dx) || !std::isfinite(d.dy) ||
      !std::isfinite(d.dz))
    return FDTD_ERR_INVALID_ARG;
  if (d.scheme < FDTD_FADI || d.scheme > FDTD_FLOD2) return FDTD_ERR_INVALID_ARG;
  if (d.precision != FDTD_F64 && d.precision != FDTD_F32) return FDTD_ERR_INVALID_ARG;
  double dt = d.dt;
  if (!(dt > 0)) {
    if (!(d.cfl > 0) || !std::isfinite(d.cfl)) return FDTD_ERR_INVALID_ARG;
    double s = 1.0 / (d.dx * d.dx) + 1.0 / (d.dy * d.dy);
    if (d.nz > 1) s += 1.0 / (d.dz * d.dz);
    dt = d.cfl / (kC0 * std::sqrt(s));
  }
  if (!std::isfinite(dt) || !(dt > 0)) return FDTD_ERR_INVALID_ARG;
  fdtd_t* h = new (std::nothrow) fdtd_s();
  if (!h) return FDTD_ERR_OOM;
  h->desc = d;
  h->nx = d.nx; h->ny = d.ny; h->nz = d.nz;
  h->dx = d.dx; h->dy = d.dy; h->dz = d.dz;
  h->dt = dt;
  h->scheme = d.scheme;
  h->prec = d.precision;
  h->esize = d.precision == FDTD_F64 ? 8 : 4;
  h->stream = (cudaStream_t)stream;
  h->pitch = std::max(((long long)(d.nx + 1) + 31) / 32 * 32, 32LL * std::max(1, pick_rows_L(d.nx)));
  h->plane = h->pitch * (d.ny + 1);
  h->count = h->plane * (d.nz + 1);
  h->pending_init = (d.scheme == FDTD_FADI || d.scheme == FDTD_FLOD2);
  build_geometry(h);
  // y/z line blocks hold every segment of a line; x rows need pitch >= 32 L
  if (pick_rows_L(d.nx) < 0) { delete h; return FDTD_ERR_UNSUPPORTED; }
  for (int ax = 0; ax < 2; ++ax) {
    const int N = ax == 0 ? d.ny : d.nz;
    StridedCfg a, b;
    if (h->prec == FDTD_F64) {
      a = choose_strided<double>(N, false, d.tune[0]);
      b = choose_strided<double>(N, true, d.tune[0]);
    } else {
      a = choose_strided<float>(N, false, d.tune[0]);
      b = choose_strided<float>(N, true, d.tune[0]);
    }
    // one configuration for both coefficient modes: the more constrained one
    if (!a.ok || !b.ok) {
      if (N >= 2) { delete h; return FDTD_ERR_UNSUPPORTED; }
    }
    h->strided_cfg[ax] = (a.lanes * a.L == b.lanes * b.L && a.lanes == b.lanes) ? a : b;
  }
  for (int c = 0; c < 6; ++c) {
    cudaError_t e = dev_malloc((void**)&h->f[c], (size_t)h->count * h->esize);
    if (e != cudaSuccess) { fdtd_destroy(h); return FDTD_ERR_OOM; }
    e = cudaMemsetAsync(h->f[c], 0, (size_t)h->count * h->esize, h->stream);
    if (e != cudaSuccess) { fdtd_destroy(h); return FDTD_ERR_CUDA; }
  }
  for (int cls = 0; cls < 3; ++cls)
    h->bytes_per_launch[cls] = 4.0 * (double)d.nx * d.ny * d.nz * (double)h->esize;
  cudaError_t e = dev_malloc((void**)&h->d_stash, sizeof(double) * fdtd::kMaxProbes);
  if (e != cudaSuccess) { fdtd_destroy(h); return FDTD_ERR_OOM; }
  e = dev_malloc((void**)&h->d_err, sizeof(int));
  if (e != cudaSuccess) { fdtd_destroy(h); return FDTD_ERR_OOM; }
  if (cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) != cudaSuccess) { fdtd_destroy(h); return FDTD_ERR_CUDA; }
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      fdtd_destroy(h);
      return FDTD_ERR_CUDA;
    }
  }
  h->use_tma = (d.tune[1] & 1) == 0;
  int rc = build_all_coefs(h);
  if (rc) { fdtd_destroy(h); return rc; }
  *out = h;
  return FDTD_OK;
}

int fdtd_destroy(fdtd_t* h) {
  if (!h) return FDTD_OK;
  cudaStreamSynchronize(h->stream);
  for (int c = 0; c < 6; ++c) {
    if (h->f[c]) cudaFree(h->f[c]);
    if (h->scratch[c]) cudaFree(h->scratch[c]);
  }
  for (auto& p : h->proc) free_coef(p);
  for (int c = 0; c < 3; ++c) {
    if (h->eps_node[c]) cudaFree(h->eps_node[c]);
    if (h->mu_node[c]) cudaFree(h->mu_node[c]);
    if (h->sig_node[c]) cudaFree(h->sig_node[c]);
  }
  if (h->d_probe) cudaFree(h->d_probe);
  if (h->d_stash) cudaFree(h->d_stash);
  if (h->d_partial) cudaFree(h->d_partial);
  if (h->d_ref_partial) cudaFree(h->d_ref_partial);
  if (h->tmp4) cudaFree(h->tmp4);
  if (h->yseq) cudaFree(h->yseq);
  if (h->d_err) cudaFree(h->d_err);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->g_run) cudaStreamSynchronize(h->g_run);
  graph_release(h);
  for (int b = 0; b < 3; ++b) {
    if (h->g_br[b]) cudaStreamDestroy(h->g_br[b]);
    if (h->g_join[b]) cudaEventDestroy(h->g_join[b]);
  }
  if (h->g_run) cudaStreamDestroy(h->g_run);
  if (h->g_in) cudaEventDestroy(h->g_in);
  if (h->g_out) cudaEventDestroy(h->g_out);
  if (h->g_fork) cudaEventDestroy(h->g_fork);
  if (h->d_srcval) cudaFree(h->d_srcval);
  if (h->d_step) cudaFree(h->d_step);
  if (h->stage) cudaFree(h->stage);
  delete h;
  return FDTD_OK;
}

int fdtd_get_dt(const fdtd_t* h, double* dt) {
  if (!h || !dt) return FDTD_ERR_INVALID_ARG;
  *dt = h->dt;
  return FDTD_OK;
}

int fdtd_steps_done(const fdtd_t* h, int64_t* n) {
  if (!h || !n) return FDTD_ERR_INVALID_ARG;
  *n = h->steps;
  return FDTD_OK;
}

int fdtd_synchronize(fdtd_t* h) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  CK(cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

int fdtd_set_material(fdtd_t* h, const double* eps, const double* mu) {
  return fdtd_set_media(h, eps, mu, nullptr);
}

int fdtd_set_order(fdtd_t* h, int order) {
  if (!h || (order != 2 && order != 4)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (h->steps > 0) return FDTD_ERR_STATE;
  if (order == h->order) return FDTD_OK;
  if (order == 4 && (h->per_node || h->mu_var || h->lossy)) return FDTD_ERR_UNSUPPORTED;
  graph_release(h);
  if (order == 4 && h->prec == FDTD_F32) CK(ensure_line4_tile_attr<float>());
  if (order == 4 && !h->tmp4) {
    CK(dev_malloc(&h->tmp4, 3 * (size_t)h->count * h->esize));
    CK(cudaMemsetAsync(h->tmp4, 0, 3 * (size_t)h->count * h->esize, h->stream));
  }
  h->order = order;
  h->output_valid = false;
  h->inv_dirty = true;
  return build_all_coefs(h);
}

int fdtd_set_media(fdtd_t* h, const double* eps, const double* mu, const double* sigma) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (h->steps > 0) return FDTD_ERR_STATE;
  const size_t nc = (size_t)h->nx * h->ny * h->nz;
  const double e0 = eps ? eps[0] : 1.0, m0 = mu ? mu[0] : 1.0, s0 = sigma ? sigma[0] : 0.0;
  bool e_uniform = true, m_uniform = true, s_uniform = true, any_loss = false;
  for (size_t q = 0; q < nc; ++q) {
    if (eps) {
      if (!(eps[q] > 0) || !std::isfinite(eps[q])) return FDTD_ERR_INVALID_ARG;
      if (eps[q] != e0) e_uniform = false;
    }
    if (mu) {
      if (!(mu[q] > 0) || !std::isfinite(mu[q])) return FDTD_ERR_INVALID_ARG;
      if (mu[q] != m0) m_uniform = false;
    }
    if (sigma) {
      if (!(sigma[q] >= 0) || !std::isfinite(sigma[q])) return FDTD_ERR_INVALID_ARG;
      if (sigma[q] != s0) s_uniform = false;
      if (sigma[q] > 0) any_loss = true;
    }
  }
  // per-node mu runs the general-media kernels, built for lines of at most
  // 256 cells along y and z and 256 along x
  if (!m_uniform && (h->nx > 256 || h->ny > 256 || h->nz > 256)) return FDTD_ERR_UNSUPPORTED;
  // fourth-order differences: uniform lossless media
  if (h->order == 4 && (!e_uniform || !m_uniform || any_loss || (h->desc.tune[1] & 2) != 0))
    return FDTD_ERR_UNSUPPORTED;
  // FADI's output relation and FLOD2's output processing solve with the loss
  // diagonal's sign flipped; they stay well conditioned (and nonsingular)
  // while sigma dt / eps <= 2 at every E sample (checked before the handle
  // changes)
  if (any_loss && (h->scheme == FDTD_FADI || h->scheme == FDTD_FLOD2)) {
    bool ok = true;
    if (e_uniform && s_uniform) {
      ok = s0 * h->dt / (kEps0 * e0) <= 2.0;
    } else {
      std::vector<double> ones, ev, sv;
      if (!eps) ones.assign(nc, 1.0);
      for (int c = 0; c < 3 && ok; ++c) {
        edge_eps(h, eps ? eps : ones.data(), c, ev);
        if (!s_uniform) edge_eps(h, sigma, c, sv);
        for (size_t q = 0; q < ev.size() && ok; ++q) {
          if (ev[q] <= 0) continue;  // row padding
          const double sg = s_uniform ? s0 : sv[q];
          if (sg * h->dt / (kEps0 * ev[q]) > 2.0) ok = false;
        }
      }
    }
    if (!ok) return FDTD_ERR_UNSUPPORTED;
  }
  graph_release(h);
  for (int c = 0; c < 3; ++c) {
    if (h->eps_node[c]) { cudaFree(h->eps_node[c]); h->eps_node[c] = nullptr; }
    if (h->mu_node[c]) { cudaFree(h->mu_node[c]); h->mu_node[c] = nullptr; }
    if (h->sig_node[c]) { cudaFree(h->sig_node[c]); h->sig_node[c] = nullptr; }
  }
  h->mu_var = !m_uniform;
  h->mu_r = h->mu_var ? 1.0 : m0;
  h->lossy = any_loss;
  const bool sig_var = any_loss && !s_uniform;
  h->sigma_u = any_loss && s_uniform ? s0 : 0.0;
  // tune[1] bit 1 keeps per-node coefficients even for a uniform eps
  h->per_node = !e_uniform || h->mu_var || sig_var || (h->desc.tune[1] & 2) != 0;
  h->eps_r = h->per_node ? 1.0 : e0;
  h->shape_tuned = false;
  int rc = FDTD_OK;
  auto release_host = [&]() {
    for (int c = 0; c < 3; ++c) {
      std::vector<double>().swap(h->eps_host[c]);
      std::vector<double>().swap(h->mu_host[c]);
      std::vector<double>().swap(h->sig_host[c]);
    }
  };
  if (h->per_node) {
    std::vector<double> ones;
    if (!eps) ones.assign(nc, 1.0);
    for (int c = 0; c < 3; ++c) {
      edge_eps(h, eps ? eps : ones.data(), c, h->eps_host[c]);
      CK(dev_malloc((void**)&h->eps_node[c], sizeof(double) * h->eps_host[c].size()));
      CK(cudaMemcpyAsync(h->eps_node[c], h->eps_host[c].data(), sizeof(double) * h->eps_host[c].size(),
                         cudaMemcpyHostToDevice, h->stream));
    }
    if (h->mu_var) {
      for (int c = 0; c < 3; ++c) {
        face_mu(h, mu, HX + c, h->mu_host[c]);
        CK(dev_malloc((void**)&h->mu_node[c], sizeof(double) * h->mu_host[c].size()));
        CK(cudaMemcpyAsync(h->mu_node[c], h->mu_host[c].data(), sizeof(double) * h->mu_host[c].size(),
                           cudaMemcpyHostToDevice, h->stream));
      }
    }
    if (sig_var) {
      // sigma at an E sample: the mean of the cells sharing its edge, as eps
      for (int c = 0; c < 3; ++c) {
        edge_eps(h, sigma, c, h->sig_host[c]);
        CK(dev_malloc((void**)&h->sig_node[c], sizeof(double) * h->sig_host[c].size()));
        CK(cudaMemcpyAsync(h->sig_node[c], h->sig_host[c].data(), sizeof(double) * h->sig_host[c].size(),
                           cudaMemcpyHostToDevice, h->stream));
      }
    }
    CK(cudaStreamSynchronize(h->stream));
  }
  rc = build_all_coefs(h);
  release_host();
  h->output_valid = false;
  h->inv_dirty = true;
  if (rc) return rc;
  return refresh_src_scale(h);
}

int fdtd_set_field(fdtd_t* h, int comp, const void* data, int on_device) {
  if (!h || !data || check_comp(comp)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  int rc;
  if ((h->scheme == FDTD_FADI || h->scheme == FDTD_FLOD2) && !h->pending_init) {
    // back to the physical field, then re-initialise on the next step
    if ((rc = physical_to_scratch(h))) return rc;
    for (int c = 0; c < 6; ++c) std::swap(h->f[c], h->scratch[c]);
    h->pending_init = true;
  }
  if ((rc = copy_in_component(h, comp, data, h->f[comp], on_device))) return rc;
  if ((rc = zero_walls(h, comp, h->f[comp]))) return rc;
  h->output_valid = false;
  h->inv_dirty = true;
  return FDTD_OK;
}

int fdtd_get_field(fdtd_t* h, int comp, void* out, int on_device) {
  if (!h || !out || check_comp(comp)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (int rc0 = check_device_flag(h)) return rc0;
  if (h->scheme == FDTD_FLOD || h->scheme == FDTD_FSS || h->pending_init)
    return copy_component(h, comp, h->f[comp], out, on_device);
  int rc = physical_to_scratch(h);
  if (rc) return rc;
  return copy_component(h, comp, h->scratch[comp], out, on_device);
}

int fdtd_get_state(fdtd_t* h, int comp, void* out, int on_device) {
  if (!h || !out || check_comp(comp)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  int rc = scheme_init(h);
  if (rc) return rc;
  return copy_component(h, comp, h->f[comp], out, on_device);
}

int fdtd_set_state(fdtd_t* h, int comp, const void* data, int on_device) {
  if (!h || !data || check_comp(comp)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  int rc = scheme_init(h);
  if (rc) return rc;
  if ((rc = copy_in_component(h, comp, data, h->f[comp], on_device))) return rc;
  if ((rc = zero_walls(h, comp, h->f[comp]))) return rc;
  h->output_valid = false;
  return FDTD_OK;
}

int fdtd_set_source(fdtd_t* h, int comp, int i, int j, int k, const double* current, int64_t count) {
  if (!h || count < 0 || (count > 0 && !current)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (count == 0) {
    h->src_comp = -1;
    h->src_current.clear();
    h->output_valid = false;
    h->inv_dirty = true;
    graph_release(h);
    return FDTD_OK;
  }
  if (comp < 0 || comp > 2) return FDTD_ERR_INVALID_ARG;
  int sx, sy, sz;
  comp_extent(comp, h->nx, h->ny, h->nz, &sx, &sy, &sz);
  if (i < 0 || j < 0 || k < 0 || i >= sx || j >= sy || k >= sz) return FDTD_ERR_INVALID_ARG;
  bool wall;
  if (comp == EX) wall = (j == 0 || j == h->ny || k == 0 || k == h->nz);
  else if (comp == EY) wall = (i == 0 || i == h->nx || k == 0 || k == h->nz);
  else wall = (i == 0 || i == h->nx || j == 0 || j == h->ny);
  if (wall) return FDTD_ERR_INVALID_ARG;
  for (int64_t q = 0; q < count; ++q)
    if (!std::isfinite(current[q])) return FDTD_ERR_INVALID_ARG;
  h->src_comp = comp;
  h->src_i = i; h->src_j = j; h->src_k = k;
  h->src_current.assign(current, current + count);
  h->output_valid = false;
  h->inv_dirty = true;
  return refresh_src_scale(h);
}

int fdtd_add_probe(fdtd_t* h, int comp, int i, int j, int k, int* id) {
  if (!h || !id || check_comp(comp)) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (h->nprobes >= fdtd::kMaxProbes) return FDTD_ERR_INVALID_ARG;
  int sx, sy, sz;
  comp_extent(comp, h->nx, h->ny, h->nz, &sx, &sy, &sz);
  if (i < 0 || j < 0 || k < 0 || i >= sx || j >= sy || k >= sz) return FDTD_ERR_INVALID_ARG;
  const int q = h->nprobes;
  h->probe_comp[q] = comp;
  h->probe_at[q] = elem_index(h, i, j, k);
  h->probe_start[q] = h->steps;
  h->nprobes++;
  *id = q;
  return FDTD_OK;
}

int fdtd_step(fdtd_t* h, int64_t nsteps) {
  if (!h || nsteps < 0) return FDTD_ERR_INVALID_ARG;
  NvtxScope range("fdtd_step");
  if (h->poisoned) return FDTD_ERR_STATE;
  if (nsteps == 0) return FDTD_OK;
  int rc = ensure_yseq(h);
  if (rc) return rc;
  rc = scheme_init(h);
  if (rc) return rc;
  if ((rc = take_invariant_ref(h))) return rc;
  if (h->per_node && !h->shape_tuned && h->desc.tune[0] == 0) {
    if ((rc = single_tune(h))) return rc;
  }
  h->shape_tuned = true;
  if ((rc = ensure_probe_capacity(h, h->steps + nsteps))) return rc;
  if (graph_usable(h)) {
    if ((rc = step_graph(h, nsteps))) return rc;
  } else {
    for (int64_t q = 0; q < nsteps; ++q)
      if ((rc = one_step(h))) return rc;
  }
  h->output_valid = false;
  return FDTD_OK;
}

int fdtd_get_probe(fdtd_t* h, int id, double* out, int64_t n) {
  if (!h || !out || id < 0 || id >= h->nprobes || n < 0) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (h->probe_start[id] + n > h->steps) return FDTD_ERR_INVALID_ARG;
  if (n == 0) return FDTD_OK;
  CK(cudaMemcpyAsync(out, h->d_probe + (size_t)id * h->probe_cap + h->probe_start[id], sizeof(double) * n,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FDTD_OK;
}

int fdtd_energy(fdtd_t* h, double out[2]) {
  NvtxScope range("fdtd_energy");
  if (!h || !out) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (int rc0 = check_device_flag(h)) return rc0;
  int rc = scheme_init(h);
  if (rc) return rc;
  if ((rc = take_invariant_ref(h))) return rc;
  if ((rc = energy(h, h->f, &out[1]))) return rc;
  if (h->scheme == FDTD_FLOD || h->scheme == FDTD_FSS) {
    out[0] = out[1];
  } else {
    if ((rc = physical_to_scratch(h))) return rc;
    if ((rc = energy(h, h->scratch, &out[0]))) return rc;
  }
  if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return FDTD_ERR_UNSTABLE;
  // growth of the invariant past its reference (runs with no source)
  if (h->inv_have && h->src_comp < 0) {
    if (h->inv_ref < 0 && (rc = energy_sum(h, h->d_ref_partial, &h->inv_ref))) return rc;
    if (out[1] > h->inv_ref * (1.0 + invariant_growth_limit(h))) return FDTD_ERR_UNSTABLE;
  }
  return FDTD_OK;
}

int fdtd_set_timing(fdtd_t* h, int enable) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  h->timing = enable != 0;
  return FDTD_OK;
}

int fdtd_get_stats(fdtd_t* h, fdtd_stats* out) {
  if (!h || !out) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  int rc = resolve_events(h);
  if (rc) return rc;
  out->launches = h->launches;
  for (int c = 0; c < 3; ++c) {
    out->timed_launches[c] = h->timed_launches[c];
    out->timed_ms[c] = h->timed_ms[c];
    out->bytes_per_launch[c] = h->bytes_per_launch[c];
  }
  return FDTD_OK;
}

int fdtd_reset_stats(fdtd_t* h) {
  if (!h) return FDTD_ERR_INVALID_ARG;
  if (h->poisoned) return FDTD_ERR_STATE;
  int rc = resolve_events(h);
  if (rc) return rc;
  h->launches = 0;
  for (int c = 0; c < 3; ++c) {
    h->timed_launches[c] = 0;
    h->timed_ms[c] = 0;
  }
  return FDTD_OK;
}

}  // extern "C"

// ===========================================================================
// Batches: many independent grids stepped together
// ===========================================================================
namespace {

// Shape of the batched launches, per line direction:
//   y, z lines: lanes (lines per tile) and L (nodes per thread; the carry
//               chains then span P = ceil(N / L) segments);
//   x lines:    warps (lines) per block.
// Grids with per-node media take any L; grids with uniform media keep the L
// their coefficient tables were built for.
struct BatchCfg {
  int lanes[2] = {16, 16};
  int L[2] = {16, 16};
  int wpb = 8;
  int xpack = 1;  // per-node x lines of up to 128 nodes share warps (8 or 16 lanes per line)
};

constexpr int kBatchBranches = 4;  // concurrent graph branches per procedure

struct BatchGroup {
  int kind = 0;             // 0 lines along y, 1 along z, 2 along x
  int L = 16, P = 1, lanes = 16, wpb = 8;
  int G = 1;                // y/z tiles per block
  int lpl = 0;              // x lines of per-node grids: lanes per line (0: one warp per line)
  int pn = 0;               // per-node media
  int ngrids = 0;
  long long nitems = 0;     // tiles (strided) or lines (x)
  void* d_params = nullptr; // PairParams<T>[ngrids]
  void* d_index = nullptr;  // BatchTile[nitems] or long long line_start[ngrids + 1]
};

}  // namespace

struct fdtd_batch_s {
  std::vector<fdtd_t*> h;
  int prec = 0, scheme = 0;
  cudaStream_t stream = nullptr;       // the handles' stream
  cudaStream_t run = nullptr;          // capture/replay stream (never the legacy default)
  cudaStream_t branch[kBatchBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
  cudaEvent_t ev_join[kBatchBranches] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<BatchGroup> groups[2];           // per procedure slot
  std::vector<const void*> bound;              // state pointers the tables were built for
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  BatchCfg cfg;
  bool tuned = false;       // cfg chosen (by the tuner, the cache or the caller)
  bool autotune = true;
  double tune_ms[3] = {0, 0, 0};  // per direction: time of the chosen shape (both procedures)
  // How a step runs: a graph of shape-uniform launches on parallel branches
  // (0), or one persistent launch per procedure taking every group's work
  // from a list (1).  mode -1: the tuner times both and keeps the faster.
  int mode = -1;
  int tuned_persistent = -1;   // the tuner's choice for the current shapes (-1: not made)
  bool persistent = false;
  double mode_ms[2] = {0, 0};  // tuned time of one step in each mode (0: not timed)
  struct Persistent {
    void* d_groups = nullptr;  // BatchGroupRef<T>[groups of the slot]
    void* d_work = nullptr;    // BatchWork[nwork]
    void* d_slots = nullptr;   // BatchSlot[] of the y/z items
    int nwork = 0, threads = 0, blocks = 0, lanes = 0, L = 0;
    size_t smem = 0;
  } pl[2];
  int* d_counter = nullptr;    // one work counter per procedure of a step
};

namespace {

void free_group_list(std::vector<BatchGroup>& gs) {
  for (auto& g : gs) {
    if (g.d_params) cudaFree(g.d_params);
    if (g.d_index) cudaFree(g.d_index);
  }
  gs.clear();
}

void free_persistent(fdtd_batch_t::Persistent (&pl)[2]) {
  for (auto& q : pl) {
    if (q.d_groups) cudaFree(q.d_groups);
    if (q.d_work) cudaFree(q.d_work);
    if (q.d_slots) cudaFree(q.d_slots);
    q = fdtd_batch_t::Persistent();
  }
}

void free_groups(fdtd_batch_t* b) {
  free_group_list(b->groups[0]);
  free_group_list(b->groups[1]);
  free_persistent(b->pl);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

#define BCK(call)                                                          \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) {                                               \
      fprintf(stderr, "fdtd batch: CUDA error: %s\n", cudaGetErrorString(_e)); \
      return _e == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA; \
    }                                                                      \
  } while (0)

template <typename T>
const void* batch_strided_fn(int lanes, int L) {
  if (lanes == 32 && L == 8) return (const void*)fdtd::proc_strided_batch_kernel<T, 32, 8>;
  if (lanes == 32 && L == 16) return (const void*)fdtd::proc_strided_batch_kernel<T, 32, 16>;
  if (lanes == 16 && L == 8) return (const void*)fdtd::proc_strided_batch_kernel<T, 16, 8>;
  if (lanes == 16 && L == 16) return (const void*)fdtd::proc_strided_batch_kernel<T, 16, 16>;
  if (lanes == 16 && L == 32) return (const void*)fdtd::proc_strided_batch_kernel<T, 16, 32>;
  if (lanes == 8 && L == 16) return (const void*)fdtd::proc_strided_batch_kernel<T, 8, 16>;
  if (lanes == 8 && L == 32) return (const void*)fdtd::proc_strided_batch_kernel<T, 8, 32>;
  return nullptr;
}

template <typename T>
bool batch_shape_ok(int N, int lanes, int L) {
  const void* fn = batch_strided_fn<T>(lanes, L);
  if (!fn) return false;
  const int P = segments(N, L, lanes);
  if (P > 32) return false;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return false;
  return P * lanes <= a.maxThreadsPerBlock;
}

// L of one grid's y/z lines under cfg: the configured L when it fits, else
// the next longer one; uniform media keep the L of their tables.
template <typename T>
int batch_grid_L(const fdtd_t* h, int kind, int N, int lanes, int Lcfg) {
  if (!h->per_node) return batch_shape_ok<T>(N, lanes, h->strided_cfg[kind].L) ? h->strided_cfg[kind].L : -1;
  for (int L : {8, 16, 32})
    if (L >= Lcfg && batch_shape_ok<T>(N, lanes, L)) return L;
  return -1;
}

// Group every pair of every grid by launch shape.  `only_kind` >= 0 keeps
// one direction (tuning); `scratch_out` writes to the handles' scratch arrays
// instead of in place (tuning runs leave the state untouched).
template <typename T>
int build_groups_t(fdtd_batch_t* b, const BatchCfg& cfg, std::vector<BatchGroup> (&out)[2], int only_kind,
                   bool scratch_out) {
  for (int slot = 0; slot < 2; ++slot) {
    struct Key {
      int kind, L, lanes, P, pn;
      std::vector<std::pair<int, int>> members;  // (grid, pair)
    };
    std::vector<Key> keys;
    for (int gi = 0; gi < (int)b->h.size(); ++gi) {
      fdtd_t* h = b->h[gi];
      const ProcCoef& P = h->proc[slot];
      for (int q = 0; q < 3; ++q) {
        const PairGeom& g = h->geom[P.op][q];
        if (g.empty()) continue;
        const int kind = g.rows ? 2 : (g.axis == AX_Y ? 0 : 1);
        if (only_kind >= 0 && kind != only_kind) continue;
        int L, lanes = 0, Pseg = 0;
        if (g.rows) {
          L = rows_L(h, g);  // the L of the grid's coefficient tables
          // per-node media take any L: short lines share a warp (8 or 16
          // lanes per line) so that every lane streams 8 nodes
          if (h->per_node && g.N <= 256 && cfg.xpack) {
            L = 8;
            lanes = g.N <= 64 ? 8 : (g.N <= 128 ? 16 : 32);
          }
        } else {
          lanes = cfg.lanes[kind];
          L = batch_grid_L<T>(h, kind, g.N, lanes, cfg.L[kind]);
          if (L < 0) return FDTD_ERR_UNSUPPORTED;
          Pseg = segments(g.N, L, lanes);
        }
        const int pn = h->per_node ? 1 : 0;  // tiles of one block share the media kind
        bool found = false;
        for (auto& k : keys)
          if (k.kind == kind && k.L == L && k.lanes == lanes && k.P == Pseg && k.pn == pn) {
            k.members.push_back({gi, q});
            found = true;
            break;
          }
        if (!found) keys.push_back({kind, L, lanes, Pseg, pn, {{gi, q}}});
      }
    }
    for (auto& k : keys) {
      BatchGroup bg;
      bg.kind = k.kind;
      bg.pn = k.pn;
      bg.L = k.L;
      bg.lanes = k.lanes;
      bg.P = k.P;
      if (bg.kind == 2) bg.lpl = k.lanes;
      if (bg.kind != 2) {
        // about 256 threads per block, within the default shared-memory limit
        const int tpt = bg.P * bg.lanes;
        bg.G = std::max(1, std::min(8, 256 / tpt));
        auto smem = [&](int G) {
          return fdtd::batch_params_bytes<T>(G) + (size_t)G * 6 * (bg.P | 1) * bg.lanes * sizeof(T);
        };
        while (bg.G > 1 && smem(bg.G) > 48 * 1024) --bg.G;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, batch_strided_fn<T>(bg.lanes, bg.L)) == cudaSuccess)
          while (bg.G > 1 && bg.G * tpt > fa.maxThreadsPerBlock) --bg.G;
      }
      bg.wpb = cfg.wpb;
      bg.ngrids = (int)k.members.size();
      std::vector<fdtd::PairParams<T>> params;
      std::vector<fdtd::BatchTile> tiles;
      std::vector<long long> starts(1, 0);
      for (int m = 0; m < bg.ngrids; ++m) {
        fdtd_t* h = b->h[k.members[m].first];
        const int q = k.members[m].second;
        const ProcCoef& P = h->proc[slot];
        const PairGeom& g = h->geom[P.op][q];
        if (scratch_out) {
          int rc = ensure_scratch(h);
          if (rc) return rc;
        }
        params.push_back(make_params<T>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, h->f, scratch_out ? h->scratch : h->f));
        if (bg.kind == 2) {
          starts.push_back(starts.back() + g.n_lines());
        } else {
          const int tx = (g.lane_hi + bg.lanes - 1) / bg.lanes;
          for (int o = 0; o < g.n_o; ++o)
            for (int bx = 0; bx < tx; ++bx) tiles.push_back({m, bx * bg.lanes, g.o_lo + o, 0});
        }
      }
      BCK(dev_malloc((void**)&bg.d_params, sizeof(fdtd::PairParams<T>) * params.size()));
      out[slot].push_back(bg);  // freed with the list from here on
      BCK(cudaMemcpy(bg.d_params, params.data(), sizeof(fdtd::PairParams<T>) * params.size(),
                     cudaMemcpyHostToDevice));
      if (bg.kind == 2) {
        bg.nitems = starts.back();
        BCK(dev_malloc((void**)&bg.d_index, sizeof(long long) * starts.size()));
        out[slot].back() = bg;
        BCK(cudaMemcpy(bg.d_index, starts.data(), sizeof(long long) * starts.size(), cudaMemcpyHostToDevice));
      } else {
        bg.nitems = (long long)tiles.size();
        BCK(dev_malloc((void**)&bg.d_index, sizeof(fdtd::BatchTile) * tiles.size()));
        out[slot].back() = bg;
        BCK(cudaMemcpy(bg.d_index, tiles.data(), sizeof(fdtd::BatchTile) * tiles.size(), cudaMemcpyHostToDevice));
      }
    }
  }
  return FDTD_OK;
}

template <typename T, int LANES, int L>
void launch_batch_strided_LL(const BatchGroup& g, cudaStream_t s) {
  const int threads = g.G * g.P * LANES;
  const size_t smem = fdtd::batch_params_bytes<T>(g.G) + (size_t)g.G * 6 * (g.P | 1) * LANES * sizeof(T);
  const unsigned blocks = (unsigned)((g.nitems + g.G - 1) / g.G);
  fdtd::proc_strided_batch_kernel<T, LANES, L><<<blocks, threads, smem, s>>>(
      (const fdtd::PairParams<T>*)g.d_params, (const fdtd::BatchTile*)g.d_index, (int)g.nitems, g.G);
}

template <typename T, int L>
void launch_batch_rows_L(const BatchGroup& g, cudaStream_t s) {
  const int wpb = g.wpb;
  fdtd::proc_rows_batch_kernel<T, L><<<(unsigned)((g.nitems + wpb - 1) / wpb), wpb * 32, 0, s>>>(
      (const fdtd::PairParams<T>*)g.d_params, (const long long*)g.d_index, g.ngrids);
}

template <typename T, int LPL>
void launch_batch_rows_pn(const BatchGroup& g, cudaStream_t s) {
  const int wpb = g.wpb;
  const long long warps = (g.nitems + (32 / LPL) - 1) / (32 / LPL);
  fdtd::proc_rows_batch_pn_kernel<T, 8, LPL><<<(unsigned)((warps + wpb - 1) / wpb), wpb * 32, 0, s>>>(
      (const fdtd::PairParams<T>*)g.d_params, (const long long*)g.d_index, g.ngrids);
}

template <typename T>
int launch_batch_group(const BatchGroup& g, cudaStream_t s) {
  if (g.kind == 2 && g.lpl > 0) {
    switch (g.lpl) {
      case 8: launch_batch_rows_pn<T, 8>(g, s); break;
      case 16: launch_batch_rows_pn<T, 16>(g, s); break;
      case 32: launch_batch_rows_pn<T, 32>(g, s); break;
      default: return FDTD_ERR_UNSUPPORTED;
    }
  } else if (g.kind == 2) {
    switch (g.L) {
      case 1: launch_batch_rows_L<T, 1>(g, s); break;
      case 2: launch_batch_rows_L<T, 2>(g, s); break;
      case 4: launch_batch_rows_L<T, 4>(g, s); break;
      case 8: launch_batch_rows_L<T, 8>(g, s); break;
      case 12: launch_batch_rows_L<T, 12>(g, s); break;
      case 16: launch_batch_rows_L<T, 16>(g, s); break;
      case 24: launch_batch_rows_L<T, 24>(g, s); break;
      case 32: launch_batch_rows_L<T, 32>(g, s); break;
      default: return FDTD_ERR_UNSUPPORTED;
    }
  } else {
    const int lanes = g.lanes, L = g.L;
    if (lanes == 32 && L == 8) launch_batch_strided_LL<T, 32, 8>(g, s);
    else if (lanes == 32 && L == 16) launch_batch_strided_LL<T, 32, 16>(g, s);
    else if (lanes == 16 && L == 8) launch_batch_strided_LL<T, 16, 8>(g, s);
    else if (lanes == 16 && L == 16) launch_batch_strided_LL<T, 16, 16>(g, s);
    else if (lanes == 16 && L == 32) launch_batch_strided_LL<T, 16, 32>(g, s);
    else if (lanes == 8 && L == 16) launch_batch_strided_LL<T, 8, 16>(g, s);
    else if (lanes == 8 && L == 32) launch_batch_strided_LL<T, 8, 32>(g, s);
    else return FDTD_ERR_UNSUPPORTED;
  }
  BCK(cudaGetLastError());
  return FDTD_OK;
}

// The persistent launches' shapes: (lanes, L) of the y/z lines (one for
// both directions) with an instantiated kernel.
// (FP64 fields: (16, 8) only; at L = 16 their solve needs more than the
// 128 registers of two 256-thread blocks per SM.)  Blocks of 256 threads:
// y/z tiles of at most 256 threads (P * lanes), i.e. lines of at most 128
// cells at L = 8 and 256 at L = 16.
constexpr int kPersistentThreads = 256;
template <typename T>
const void* persistent_fn(int lanes, int L) {
  if (lanes == 16 && L == 8) return (const void*)fdtd::proc_batch_persistent_kernel<T, 16, 8>;
  if constexpr (sizeof(T) == 4)
    if (lanes == 16 && L == 16) return (const void*)fdtd::proc_batch_persistent_kernel<T, 16, 16>;
  return nullptr;
}

// Work lists of the persistent launches, one per procedure slot, from the
// groups built for the same shapes.  The y/z tiles of every group are packed
// into items of kPersistentThreads threads, best fit by free warps, largest
// tiles first; the threads an item leaves over form its spare slot.
// FDTD_ERR_UNSUPPORTED when the groups do not fit one persistent kernel:
// y and z lines of different (lanes, L), a shape without an instantiated
// kernel, uniform media (their y/z tiles may read coefficient tables, which
// a spare slot of another segment count must not), or x lines not packed.
template <typename T>
int build_persistent_t(const std::vector<BatchGroup> (&gs)[2], fdtd_batch_t::Persistent (&out)[2]) {
  int lanes = 0, L = 0, maxtpt = 32;
  for (int slot = 0; slot < 2; ++slot)
    for (const auto& g : gs[slot]) {
      if (!g.pn) return FDTD_ERR_UNSUPPORTED;
      if (g.kind == 2) {
        if (g.lpl != 8 && g.lpl != 16 && g.lpl != 32) return FDTD_ERR_UNSUPPORTED;
        continue;
      }
      if (lanes == 0) {
        lanes = g.lanes;
        L = g.L;
      }
      if (g.lanes != lanes || g.L != L) return FDTD_ERR_UNSUPPORTED;
      maxtpt = std::max(maxtpt, g.P * g.lanes);
    }
  if (lanes == 0) {  // no y/z lines at all: any instantiated shape serves the x lines
    lanes = 16;
    L = 8;
  }
  const void* fn = persistent_fn<T>(lanes, L);
  if (!fn) return FDTD_ERR_UNSUPPORTED;
  const int threads = kPersistentThreads;
  if (maxtpt > threads) return FDTD_ERR_UNSUPPORTED;
  const int warps = threads / 32;
  cudaFuncAttributes fa;
  BCK(cudaFuncGetAttributes(&fa, fn));
  if (threads > fa.maxThreadsPerBlock) return FDTD_ERR_UNSUPPORTED;
  int dev = 0, nsm = 1;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  size_t smem = 0;
  for (int slot = 0; slot < 2; ++slot) {
    fdtd_batch_t::Persistent& q = out[slot];
    std::vector<fdtd::BatchGroupRef<T>> refs;
    std::vector<fdtd::BatchWork> work, work_x;
    std::vector<fdtd::BatchSlot> slots;
    // y/z groups by tile size, largest first
    std::vector<int> order;
    for (size_t gi = 0; gi < gs[slot].size(); ++gi) {
      const BatchGroup& g = gs[slot][gi];
      fdtd::BatchGroupRef<T> r{};
      r.params = (const fdtd::PairParams<T>*)g.d_params;
      r.index = g.d_index;
      r.nitems = g.nitems;
      r.ngrids = g.ngrids;
      if (g.kind == 2) {
        r.kind = 1;
        r.lpl = g.lpl;
        const long long nw = (g.nitems + (32 / g.lpl) - 1) / (32 / g.lpl);
        for (long long w0 = 0; w0 < nw; w0 += warps) work_x.push_back({(int)gi, 0, w0});
      } else {
        r.kind = 0;
        r.P = g.P;
        order.push_back((int)gi);
      }
      refs.push_back(r);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return gs[slot][a].P > gs[slot][b].P; });
    struct Item {
      std::vector<fdtd::BatchSlot> s;
      int free;
    };
    std::vector<Item> items;
    std::vector<std::vector<int>> open(warps + 1);  // items by free warps
    for (int gi : order) {
      const BatchGroup& g = gs[slot][gi];
      const int need = g.P * g.lanes / 32;
      for (long long t = 0; t < g.nitems; ++t) {
        int it = -1;
        for (int f = need; f < warps && it < 0; ++f)
          if (!open[f].empty()) {
            it = open[f].back();
            open[f].pop_back();
          }
        if (it < 0) {
          it = (int)items.size();
          items.push_back({{}, warps});
        }
        Item& m = items[it];
        m.s.push_back({gi, (int)t, (warps - m.free) * 32, need * 32, 0, 0});
        m.free -= need;
        if (m.free > 0) open[m.free].push_back(it);
      }
    }
    for (Item& m : items) {
      if (m.free > 0) m.s.push_back({m.s[0].group, -1, (warps - m.free) * 32, m.free * 32, 0, 0});
      int coff = 0;
      for (auto& b : m.s) {
        b.coff = coff;
        coff += 6 * ((b.tpt / lanes) | 1) * lanes;
      }
      smem = std::max(smem, fdtd::batch_params_bytes<T>((int)m.s.size()) + (size_t)coff * sizeof(T));
      work.push_back({-1, (int)m.s.size(), (long long)slots.size()});
      slots.insert(slots.end(), m.s.begin(), m.s.end());
    }
    work.insert(work.end(), work_x.begin(), work_x.end());
    q.threads = threads;
    q.lanes = lanes;
    q.L = L;
    q.nwork = (int)work.size();
    if (!refs.empty()) {
      BCK(dev_malloc(&q.d_groups, sizeof(fdtd::BatchGroupRef<T>) * refs.size()));
      BCK(cudaMemcpy(q.d_groups, refs.data(), sizeof(fdtd::BatchGroupRef<T>) * refs.size(), cudaMemcpyHostToDevice));
    }
    if (!work.empty()) {
      BCK(dev_malloc(&q.d_work, sizeof(fdtd::BatchWork) * work.size()));
      BCK(cudaMemcpy(q.d_work, work.data(), sizeof(fdtd::BatchWork) * work.size(), cudaMemcpyHostToDevice));
    }
    if (!slots.empty()) {
      BCK(dev_malloc(&q.d_slots, sizeof(fdtd::BatchSlot) * slots.size()));
      BCK(cudaMemcpy(q.d_slots, slots.data(), sizeof(fdtd::BatchSlot) * slots.size(), cudaMemcpyHostToDevice));
    }
  }
  if (smem > 227 * 1024) return FDTD_ERR_UNSUPPORTED;
  if (smem > 48 * 1024) BCK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  if (per_sm < 1) return FDTD_ERR_UNSUPPORTED;
  for (auto& q : out) {
    q.smem = smem;
    q.blocks = (int)std::min<long long>(std::max(1, q.nwork), (long long)nsm * per_sm);
  }
  return FDTD_OK;
}

template <typename T>
int launch_persistent(const fdtd_batch_t::Persistent& q, int* counter, cudaStream_t s) {
  if (q.nwork == 0) return FDTD_OK;
  BCK(cudaMemsetAsync(counter, 0, sizeof(int), s));
  const auto* groups = (const fdtd::BatchGroupRef<T>*)q.d_groups;
  const auto* work = (const fdtd::BatchWork*)q.d_work;
  const auto* slots = (const fdtd::BatchSlot*)q.d_slots;
  if (q.lanes == 16 && q.L == 8) {
    fdtd::proc_batch_persistent_kernel<T, 16, 8><<<q.blocks, q.threads, q.smem, s>>>(groups, work, slots, q.nwork,
                                                                                      counter);
  } else if constexpr (sizeof(T) == 4) {
    if (q.lanes == 16 && q.L == 16)
      fdtd::proc_batch_persistent_kernel<T, 16, 16><<<q.blocks, q.threads, q.smem, s>>>(groups, work, slots,
                                                                                         q.nwork, counter);
    else
      return FDTD_ERR_UNSUPPORTED;
  } else {
    return FDTD_ERR_UNSUPPORTED;
  }
  BCK(cudaGetLastError());
  return FDTD_OK;
}

// One time step of every grid: the scheme's procedure sequence.  The groups
// of one procedure write disjoint arrays, so they fork onto parallel
// branches; the next procedure starts when all of them have joined.  In
// persistent mode each procedure is one launch (after the reset of its work
// counter).
template <typename T>
int batch_one_step_with(fdtd_batch_t* b, const std::vector<BatchGroup> (&groups)[2],
                        const fdtd_batch_t::Persistent (&pl)[2], bool persistent) {
  static const int seq_fss[3] = {0, 1, 0};
  static const int seq_two[2] = {0, 1};
  const int* seq = b->scheme == FDTD_FSS ? seq_fss : seq_two;
  const int n = b->scheme == FDTD_FSS ? 3 : 2;
  if (persistent) {
    for (int k = 0; k < n; ++k) {
      int rc = launch_persistent<T>(pl[seq[k]], b->d_counter + k, b->run);
      if (rc) return rc;
    }
    return FDTD_OK;
  }
  for (int k = 0; k < n; ++k) {
    const auto& gs = groups[seq[k]];
    const int nb = std::min<int>(kBatchBranches, (int)gs.size());
    BCK(cudaEventRecord(b->ev_fork, b->run));
    for (int i = 0; i < nb; ++i) BCK(cudaStreamWaitEvent(b->branch[i], b->ev_fork, 0));
    for (size_t gi = 0; gi < gs.size(); ++gi) {
      int rc = launch_batch_group<T>(gs[gi], b->branch[gi % nb]);
      if (rc) return rc;
    }
    for (int i = 0; i < nb; ++i) {
      BCK(cudaEventRecord(b->ev_join[i], b->branch[i]));
      BCK(cudaStreamWaitEvent(b->run, b->ev_join[i], 0));
    }
  }
  return FDTD_OK;
}

template <typename T>
int batch_one_step(fdtd_batch_t* b) {
  return batch_one_step_with<T>(b, b->groups, b->pl, b->persistent);
}

// ---------------------------------------------------------------------------
// Tuner: per direction, time the candidate launch shapes on the batch's own
// data (both procedures, out of place into scratch) and keep the fastest.
// Results are cached per (device, precision, scheme, grid list) for the
// process, and in the file named by FDTD_TUNE_CACHE when that is set.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
// every tuner's results: key -> five shape numbers (see the key makers)
using TuneVal = std::array<int, 6>;
std::map<std::string, TuneVal> g_tune_cache;

std::string device_name();

std::string batch_key(const fdtd_batch_t* b) {
  const std::string name = device_name();
  std::string s = "batch|" + name + "|p" + std::to_string(b->prec) + "|s" + std::to_string(b->scheme);
  for (const fdtd_t* h : b->h)
    s += "|" + std::to_string(h->nx) + "x" + std::to_string(h->ny) + "x" + std::to_string(h->nz) +
         (h->per_node ? "n" : "u");
  // long keys are folded to a hash (FNV-1a) after the device and precision
  if (s.size() > 200) {
    uint64_t x = 1469598103934665603ull;
    for (char c : s) x = (x ^ (unsigned char)c) * 1099511628211ull;
    char buf[32];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)x);
    s = "batch|" + name + "|p" + std::to_string(b->prec) + "|n" + std::to_string(b->h.size()) + "|" + buf;
  }
  return s;
}

// The file named by FDTD_TUNE_CACHE (when set) is read once per process and
// every new result is appended: "key v0 v1 v2 v3 v4" per line.
void tune_cache_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = getenv("FDTD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[512];
  TuneVal v;
  while (fscanf(f, "%511s %d %d %d %d %d %d", key, &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 7)
    g_tune_cache[key] = v;
  fclose(f);
}

bool tune_cache_get(const std::string& key, TuneVal* v) {
  tune_cache_load();
  auto it = g_tune_cache.find(key);
  if (it == g_tune_cache.end()) return false;
  *v = it->second;
  return true;
}

void tune_cache_put(const std::string& key, const TuneVal& v) {
  g_tune_cache[key] = v;
  const char* path = getenv("FDTD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3], v[4], v[5]);
  fclose(f);
}

// Time of one direction's launches for both procedures under cfg (ms, best
// of `reps`), or a negative value when the shape does not apply.
template <typename T>
double time_direction(fdtd_batch_t* b, const BatchCfg& cfg, int kind, int reps) {
  std::vector<BatchGroup> gs[2];
  if (build_groups_t<T>(b, cfg, gs, kind, true) != FDTD_OK) {
    free_group_list(gs[0]);
    free_group_list(gs[1]);
    cudaGetLastError();
    return -1.0;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  bool ok = true;
  for (int r = 0; r < reps + 1 && ok; ++r) {  // the first pass warms up
    cudaEventRecord(e0, b->run);
    for (int slot = 0; slot < 2 && ok; ++slot)
      for (const auto& g : gs[slot])
        if (launch_batch_group<T>(g, b->run) != FDTD_OK) ok = false;
    cudaEventRecord(e1, b->run);
    if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_group_list(gs[0]);
  free_group_list(gs[1]);
  return ok ? best : -1.0;
}

// Time of one step (ms, best of `reps` replays of a captured one-step graph,
// writing scratch) in each mode under cfg; a negative value when the mode
// does not apply.
template <typename T>
int time_step_modes(fdtd_batch_t* b, const BatchCfg& cfg, int reps, double out[2], bool launches = true) {
  out[0] = out[1] = -1.0;
  std::vector<BatchGroup> gs[2];
  fdtd_batch_t::Persistent pl[2];
  int rc = build_groups_t<T>(b, cfg, gs, -1, true);
  const bool have_pl = rc == FDTD_OK && build_persistent_t<T>(gs, pl) == FDTD_OK;
  cudaGetLastError();
  for (int mode = launches ? 0 : 1; mode < 2 && rc == FDTD_OK; ++mode) {
    if (mode == 1 && !have_pl) break;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    if (cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
    const int rs = batch_one_step_with<T>(b, gs, pl, mode == 1);
    const cudaError_t e = cudaStreamEndCapture(b->run, &g);
    if (rs != FDTD_OK || e != cudaSuccess || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      continue;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    bool ok = true;
    for (int r = 0; r < reps + 1 && ok; ++r) {  // the first replay warms up
      cudaEventRecord(e0, b->run);
      if (cudaGraphLaunch(ex, b->run) != cudaSuccess) ok = false;
      cudaEventRecord(e1, b->run);
      if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    if (ok) out[mode] = best;
  }
  free_group_list(gs[0]);
  free_group_list(gs[1]);
  free_persistent(pl);
  BCK(cudaGetLastError());
  return rc;
}

std::string batch_mode_key(const fdtd_batch_t* b) {
  const BatchCfg& c = b->cfg;
  return batch_key(b) + "|mode|" + std::to_string(c.lanes[0]) + "," + std::to_string(c.L[0]) + "," +
         std::to_string(c.lanes[1]) + "," + std::to_string(c.L[1]) + "," + std::to_string(c.wpb) + "," +
         std::to_string(c.xpack);
}

// The tuner's choice between the two modes (cached like the shapes): the
// graph of launches with the current shapes against the persistent launches
// with the current shapes, when they fit one persistent kernel, and with
// each built persistent shape on both y and z; a persistent win brings its
// shapes along.
template <typename T>
int batch_tune_mode_t(fdtd_batch_t* b) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const std::string key = batch_mode_key(b);
  TuneVal v;
  auto take = [&](int pers, int Ly, int Lz) {
    b->tuned_persistent = pers;
    if (pers) {
      b->cfg.lanes[0] = b->cfg.lanes[1] = 16;
      b->cfg.L[0] = Ly;
      b->cfg.L[1] = Lz;
      b->cfg.xpack = 1;
    }
  };
  if (tune_cache_get(key, &v)) {
    b->mode_ms[0] = v[1] * 1e-3;
    b->mode_ms[1] = v[2] * 1e-3;
    take(v[0], v[3], v[4]);
    return FDTD_OK;
  }
  BCK(cudaEventRecord(b->ev_in, b->stream));
  BCK(cudaStreamWaitEvent(b->run, b->ev_in, 0));
  double ms[2];
  int rc = time_step_modes<T>(b, b->cfg, 5, ms);
  if (rc) return rc;
  double best = ms[1];
  BatchCfg pick = b->cfg;
  for (int L : {8, 16}) {
    BatchCfg c = b->cfg;
    c.lanes[0] = c.lanes[1] = 16;
    c.L[0] = c.L[1] = L;
    c.xpack = 1;
    if (!persistent_fn<T>(16, L)) continue;
    if (c.lanes[0] == b->cfg.lanes[0] && c.lanes[1] == b->cfg.lanes[1] && c.L[0] == b->cfg.L[0] &&
        c.L[1] == b->cfg.L[1] && c.xpack == b->cfg.xpack)
      continue;  // timed above
    double m2[2];
    if ((rc = time_step_modes<T>(b, c, 5, m2, false))) return rc;
    if (m2[1] > 0 && (best < 0 || m2[1] < best)) {
      best = m2[1];
      pick = c;
    }
  }
  b->mode_ms[0] = ms[0] > 0 ? ms[0] : 0;
  b->mode_ms[1] = best > 0 ? best : 0;
  const int pers = (best > 0 && (ms[0] < 0 || best < ms[0])) ? 1 : 0;
  take(pers, pick.L[0], pick.L[1]);
  tune_cache_put(key, {pers, (int)std::lround(b->mode_ms[0] * 1e3), (int)std::lround(b->mode_ms[1] * 1e3),
                       pick.L[0], pick.L[1], 0});
  return FDTD_OK;
}

template <typename T>
int batch_tune_t(fdtd_batch_t* b) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const std::string key = batch_key(b);
  TuneVal v;
  if (tune_cache_get(key, &v)) {
    b->cfg.lanes[0] = v[0];
    b->cfg.L[0] = v[1];
    b->cfg.lanes[1] = v[2];
    b->cfg.L[1] = v[3];
    b->cfg.wpb = v[4];
    b->cfg.xpack = v[5];
    b->tuned = true;
    return FDTD_OK;
  }
  // the tuning runs read the state and write scratch: order after the
  // handles' earlier work
  BCK(cudaEventRecord(b->ev_in, b->stream));
  BCK(cudaStreamWaitEvent(b->run, b->ev_in, 0));
  static const int c32[][2] = {{16, 8}, {16, 16}, {16, 32}, {32, 8}, {32, 16}};
  static const int c64[][2] = {{16, 8}, {16, 16}, {16, 32}, {8, 16}, {8, 32}};
  const int(*cand)[2] = sizeof(T) == 8 ? c64 : c32;
  BatchCfg cfg = b->cfg;
  for (int kind = 0; kind < 2; ++kind) {
    double best = -1;
    BatchCfg pick = cfg;
    for (int q = 0; q < 5; ++q) {
      BatchCfg t = cfg;
      t.lanes[kind] = cand[q][0];
      t.L[kind] = cand[q][1];
      const double ms = time_direction<T>(b, t, kind, 3);
      if (ms >= 0 && (best < 0 || ms < best)) {
        best = ms;
        pick = t;
      }
    }
    if (best < 0) return FDTD_ERR_UNSUPPORTED;
    cfg = pick;
    b->tune_ms[kind] = best;
  }
  {
    double best = -1;
    int pick = cfg.wpb, pick_pack = cfg.xpack;
    for (int xpack : {1, 0})
      for (int wpb : {4, 8, 16}) {
        BatchCfg t = cfg;
        t.wpb = wpb;
        t.xpack = xpack;
        const double ms = time_direction<T>(b, t, 2, 3);
        if (ms >= 0 && (best < 0 || ms < best)) {
          best = ms;
          pick = wpb;
          pick_pack = xpack;
        }
      }
    cfg.wpb = pick;
    cfg.xpack = pick_pack;
    b->tune_ms[2] = best < 0 ? 0 : best;
  }
  BCK(cudaGetLastError());
  b->cfg = cfg;
  b->tuned = true;
  tune_cache_put(key, {cfg.lanes[0], cfg.L[0], cfg.lanes[1], cfg.L[1], cfg.wpb, cfg.xpack});
  return FDTD_OK;
}

int batch_prepare(fdtd_batch_t* b) {
  for (fdtd_t* h : b->h) {
    int rc = scheme_init(h);
    if (rc) return rc;
    if ((rc = take_invariant_ref(h))) return rc;
  }
  if (!b->tuned) {
    if (b->autotune) {
      int rc = b->prec == FDTD_F64 ? batch_tune_t<double>(b) : batch_tune_t<float>(b);
      if (rc) return rc;
    }
    b->tuned = true;
    b->tuned_persistent = -1;
    b->bound.clear();
  }
  if (!b->d_counter) BCK(dev_malloc((void**)&b->d_counter, 3 * sizeof(int)));
  if (b->mode == -1 && b->tuned_persistent < 0) {
    int rc = b->prec == FDTD_F64 ? batch_tune_mode_t<double>(b) : batch_tune_mode_t<float>(b);
    if (rc) return rc;
  }
  const bool want = b->mode == 1 || (b->mode == -1 && b->tuned_persistent == 1);
  std::vector<const void*> ptrs;
  for (fdtd_t* h : b->h)
    for (int c = 0; c < 6; ++c) ptrs.push_back(h->f[c]);
  if (ptrs == b->bound && !b->groups[0].empty() && want == b->persistent) return FDTD_OK;
  free_groups(b);
  int rc = b->prec == FDTD_F64 ? build_groups_t<double>(b, b->cfg, b->groups, -1, false)
                               : build_groups_t<float>(b, b->cfg, b->groups, -1, false);
  b->persistent = false;
  if (!rc && want) {
    rc = b->prec == FDTD_F64 ? build_persistent_t<double>(b->groups, b->pl)
                             : build_persistent_t<float>(b->groups, b->pl);
    b->persistent = rc == FDTD_OK;
  }
  if (rc) {
    free_groups(b);
    return rc;
  }
  b->bound = ptrs;
  return FDTD_OK;
}

// ---------------------------------------------------------------------------
// Single handles with per-node media: their y/z kernels take any (lanes, L)
// (the per-node solve has no L-dependent tables).  At the first step each
// candidate is timed on the handle's own data (both procedures, out of
// place into scratch) and the fastest kept; cached per (device, precision,
// scheme, grid) for the process.
// ---------------------------------------------------------------------------
std::string device_name() {
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "?";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  return name;
}

template <typename T>
bool strided_ok(int N, bool pn, int lanes, int L) {
  const void* fn = strided_fn_rt<T>(pn, lanes, L);
  if (!fn) return false;
  const int P = segments(N, L, lanes);
  if (P > 32) return false;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return false;
  return P * lanes <= a.maxThreadsPerBlock;
}

template <typename T>
double time_axis(fdtd_t* h, int ax, const StridedCfg& c, int reps) {
  if (ensure_scratch(h) != FDTD_OK) return -1.0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0;
  }
  double best = 1e30;
  bool ok = true;
  for (int r = 0; r < reps + 1 && ok; ++r) {  // the first pass warms up
    cudaEventRecord(e0, h->stream);
    for (int slot = 0; slot < 2; ++slot) {
      const ProcCoef& P = h->proc[slot];
      for (int q = 0; q < 3; ++q) {
        const PairGeom& g = h->geom[P.op][q];
        if (g.empty() || g.rows || (g.axis == AX_Y ? 0 : 1) != ax) continue;
        fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, h->f, h->scratch);
        launch_strided<T>(h, g, p, true, c.lanes, c.L);
      }
    }
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) ok = false;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0) best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? best : -1.0;
}

template <typename T>
int single_tune_t(fdtd_t* h) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const std::string key = "grid|" + device_name() + "|p" + std::to_string(h->prec) + "|s" +
                          std::to_string(h->scheme) + "|" + std::to_string(h->nx) + "x" + std::to_string(h->ny) +
                          "x" + std::to_string(h->nz);
  TuneVal v;
  if (tune_cache_get(key, &v) && strided_ok<T>(std::max(h->ny, 2), true, v[0], v[1]) &&
      strided_ok<T>(std::max(h->nz, 2), true, v[2], v[3])) {
    h->strided_cfg[0] = {true, v[0], v[1]};
    h->strided_cfg[1] = {true, v[2], v[3]};
    return FDTD_OK;
  }
  static const int c32[][2] = {{32, 8}, {32, 16}, {16, 8}, {16, 16}, {16, 32}};
  static const int c64[][2] = {{16, 8}, {16, 16}, {8, 16}, {8, 32}, {16, 32}};
  const int(*cand)[2] = sizeof(T) == 8 ? c64 : c32;
  for (int ax = 0; ax < 2; ++ax) {
    const int N = ax == 0 ? h->ny : h->nz;
    if (N < 2) continue;
    double best = -1;
    StridedCfg pick = h->strided_cfg[ax];
    for (int q = 0; q < 5; ++q) {
      if (!strided_ok<T>(N, true, cand[q][0], cand[q][1])) continue;
      StridedCfg c;
      c.ok = true;
      c.lanes = cand[q][0];
      c.L = cand[q][1];
      const double ms = time_axis<T>(h, ax, c, 3);
      if (ms >= 0 && (best < 0 || ms < best)) {
        best = ms;
        pick = c;
      }
    }
    h->strided_cfg[ax] = pick;
  }
  h->output_valid = false;  // scratch was written
  CK(cudaGetLastError());
  tune_cache_put(key, {h->strided_cfg[0].lanes, h->strided_cfg[0].L, h->strided_cfg[1].lanes,
                       h->strided_cfg[1].L, 0, 0});
  return FDTD_OK;
}

int single_tune(fdtd_t* h) { return h->prec == FDTD_F64 ? single_tune_t<double>(h) : single_tune_t<float>(h); }

}  // namespace

extern "C" {

int fdtd_batch_create(fdtd_t* const* handles, int count, void* stream, fdtd_batch_t** out) {
  if (!handles || count < 1 || !out) return FDTD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    fdtd_t* h = handles[i];
    if (!h) return FDTD_ERR_INVALID_ARG;
    if (h->poisoned) return FDTD_ERR_STATE;
    if (h->scheme != handles[0]->scheme || h->prec != handles[0]->prec) return FDTD_ERR_INVALID_ARG;
    if (h->stream != (cudaStream_t)stream) return FDTD_ERR_INVALID_ARG;
    if (h->src_comp >= 0 || h->nprobes > 0 || h->mu_var || h->order != 2) return FDTD_ERR_UNSUPPORTED;
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) return FDTD_ERR_INVALID_ARG;
  }
  fdtd_batch_t* b = new (std::nothrow) fdtd_batch_s();
  if (!b) return FDTD_ERR_OOM;
  b->h.assign(handles, handles + count);
  b->prec = handles[0]->prec;
  b->scheme = handles[0]->scheme;
  b->stream = (cudaStream_t)stream;
  bool ok = cudaStreamCreateWithFlags(&b->run, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < kBatchBranches && ok; ++i)
    ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    fdtd_batch_destroy(b);
    return FDTD_ERR_CUDA;
  }
  if (b->prec == FDTD_F64) {
    b->cfg.lanes[0] = b->cfg.lanes[1] = 16;
  }
  *out = b;
  return FDTD_OK;
}

int fdtd_batch_destroy(fdtd_batch_t* b) {
  if (!b) return FDTD_OK;
  if (b->run) cudaStreamSynchronize(b->run);
  cudaStreamSynchronize(b->stream);
  free_groups(b);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int i = 0; i < kBatchBranches; ++i) {
    if (b->branch[i]) cudaStreamDestroy(b->branch[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->run) cudaStreamDestroy(b->run);
  delete b;
  return FDTD_OK;
}

int fdtd_batch_step(fdtd_batch_t* b, int64_t nsteps) {
  if (!b || nsteps < 0) return FDTD_ERR_INVALID_ARG;
  NvtxScope range("fdtd_batch_step");
  for (fdtd_t* h : b->h) {
    if (h->poisoned) return FDTD_ERR_STATE;
    if (h->src_comp >= 0 || h->nprobes > 0) return FDTD_ERR_UNSUPPORTED;
  }
  if (nsteps == 0) return FDTD_OK;
  int rc = batch_prepare(b);
  if (rc) return rc;
  if (!b->exec) {
    // one step of every grid, captured once as a CUDA graph and replayed
    BCK(cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal));
    rc = b->prec == FDTD_F64 ? batch_one_step<double>(b) : batch_one_step<float>(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->run, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    BCK(e);
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  // order after the handles' earlier work, and their later work after this
  BCK(cudaEventRecord(b->ev_in, b->stream));
  BCK(cudaStreamWaitEvent(b->run, b->ev_in, 0));
  for (int64_t k = 0; k < nsteps; ++k) BCK(cudaGraphLaunch(b->exec, b->run));
  BCK(cudaEventRecord(b->ev_out, b->run));
  BCK(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  for (fdtd_t* h : b->h) {
    h->steps += nsteps;
    h->output_valid = false;
  }
  return FDTD_OK;
}

int fdtd_batch_launches(const fdtd_batch_t* b, int64_t* per_step) {
  if (!b || !per_step) return FDTD_ERR_INVALID_ARG;
  const int n = b->scheme == FDTD_FSS ? 3 : 2;
  const int seq[3] = {0, 1, 0};
  long long c = 0;
  for (int k = 0; k < n; ++k)
    c += b->persistent ? (b->pl[seq[k]].nwork > 0 ? 1 : 0) : (long long)b->groups[seq[k]].size();
  *per_step = c;
  return FDTD_OK;
}

int fdtd_batch_set_mode(fdtd_batch_t* b, int mode) {
  if (!b || mode < -1 || mode > 1) return FDTD_ERR_INVALID_ARG;
  if (mode == b->mode) return FDTD_OK;
  b->mode = mode;
  free_groups(b);
  b->bound.clear();
  return FDTD_OK;
}

int fdtd_batch_get_mode(const fdtd_batch_t* b, int32_t* persistent, double step_ms[2]) {
  if (!b || !persistent) return FDTD_ERR_INVALID_ARG;
  *persistent = b->persistent ? 1 : 0;
  if (step_ms) {
    step_ms[0] = b->mode_ms[0];
    step_ms[1] = b->mode_ms[1];
  }
  return FDTD_OK;
}

int fdtd_batch_get_config(const fdtd_batch_t* b, int32_t cfg[6], double tune_ms[3]) {
  if (!b || !cfg) return FDTD_ERR_INVALID_ARG;
  cfg[0] = b->cfg.lanes[0];
  cfg[1] = b->cfg.L[0];
  cfg[2] = b->cfg.lanes[1];
  cfg[3] = b->cfg.L[1];
  cfg[4] = b->cfg.wpb;
  cfg[5] = b->cfg.xpack;
  if (tune_ms)
    for (int k = 0; k < 3; ++k) tune_ms[k] = b->tune_ms[k];
  return FDTD_OK;
}

int fdtd_batch_set_config(fdtd_batch_t* b, const int32_t* cfg) {
  if (!b) return FDTD_ERR_INVALID_ARG;
  if (!cfg) {  // back to automatic: tune again before the next step
    b->autotune = true;
    b->tuned = false;
    free_groups(b);
    b->bound.clear();
    return FDTD_OK;
  }
  for (int k = 0; k < 2; ++k) {
    const int lanes = cfg[2 * k], L = cfg[2 * k + 1];
    const void* fn = b->prec == FDTD_F64 ? batch_strided_fn<double>(lanes, L) : batch_strided_fn<float>(lanes, L);
    if (!fn) return FDTD_ERR_INVALID_ARG;
  }
  if (cfg[4] != 4 && cfg[4] != 8 && cfg[4] != 16) return FDTD_ERR_INVALID_ARG;
  if (cfg[5] != 0 && cfg[5] != 1) return FDTD_ERR_INVALID_ARG;
  b->cfg.lanes[0] = cfg[0];
  b->cfg.L[0] = cfg[1];
  b->cfg.lanes[1] = cfg[2];
  b->cfg.L[1] = cfg[3];
  b->cfg.wpb = cfg[4];
  b->cfg.xpack = cfg[5];
  b->autotune = false;
  b->tuned = true;
  b->tuned_persistent = -1;
  free_groups(b);
  b->bound.clear();
  return FDTD_OK;
}

}  // extern "C"

// ===========================================================================
// Reverse mode: gradient of a probe-energy objective with respect to eps
// ===========================================================================
namespace {

struct AdjCfg {
  bool ok = false;
  int lanes = 16, L = 16;
};

template <typename T>
const void* adj_strided_fn(int lanes, int L) {
  if (lanes == 32 && L == 8) return (const void*)fdtd::adj_strided_kernel<T, 32, 8>;
  if (lanes == 32 && L == 16) return (const void*)fdtd::adj_strided_kernel<T, 32, 16>;
  if (lanes == 16 && L == 8) return (const void*)fdtd::adj_strided_kernel<T, 16, 8>;
  if (lanes == 16 && L == 16) return (const void*)fdtd::adj_strided_kernel<T, 16, 16>;
  if (lanes == 16 && L == 32) return (const void*)fdtd::adj_strided_kernel<T, 16, 32>;
  if (lanes == 8 && L == 32) return (const void*)fdtd::adj_strided_kernel<T, 8, 32>;
  return nullptr;
}

// Segment layout of the adjoint y/z kernel for lines of N cells (the
// per-node solve builds its carries on the fly, so any L works).
template <typename T>
AdjCfg adj_strided_cfg(int N) {
  static const int c32[][2] = {{32, 16}, {32, 8}, {16, 16}, {16, 32}, {8, 32}};
  static const int c64[][2] = {{16, 16}, {16, 8}, {16, 32}, {8, 32}, {8, 32}};
  const int(*cand)[2] = sizeof(T) == 8 ? c64 : c32;
  AdjCfg best;
  for (int q = 0; q < 5; ++q) {
    const int lanes = cand[q][0], L = cand[q][1];
    const int P = segments(N, L, lanes);
    if (P > 32) continue;
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, adj_strided_fn<T>(lanes, L)) != cudaSuccess) continue;
    if (P * lanes > a.maxThreadsPerBlock) continue;
    best.ok = true;
    best.lanes = lanes;
    best.L = L;
    return best;
  }
  return best;
}

template <typename T, int LANES, int L>
void launch_adj_strided_L(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p,
                          const fdtd::AdjExtra<T>& x) {
  const int P = segments(g.N, L, LANES);
  dim3 grid((unsigned)((g.lane_hi + LANES - 1) / LANES), (unsigned)g.n_o);
  const size_t smem = 6 * (size_t)(P | 1) * LANES * sizeof(T);
  fdtd::adj_strided_kernel<T, LANES, L><<<grid, P * LANES, smem, h->stream>>>(p, x);
}

template <typename T, int L>
void launch_adj_rows_L(const fdtd_t* h, const PairGeom& g, const fdtd::PairParams<T>& p,
                       const fdtd::AdjExtra<T>& x) {
  const int wpb = 8;
  const unsigned blocks = (unsigned)((g.n_lines() + wpb - 1) / wpb);
  fdtd::adj_rows_kernel<T, L><<<blocks, wpb * 32, 0, h->stream>>>(p, x);
}

}  // namespace

struct fdtd_adj_s {
  fdtd_t* h = nullptr;
  long long nsteps = 0;
  int every = 1, nseg = 0;
  int nprobe = 0;
  long long* d_probe_at = nullptr;
  int* d_probe_comp = nullptr;
  double* d_stash = nullptr;
  double* d_acc = nullptr;
  double* d_cell = nullptr;
  void* ckpt = nullptr;     // nseg x 6 state arrays
  void* tape = nullptr;     // 2 every x 3 records D (per procedure, per E component) of one segment
  double* d_wrec = nullptr; // every x nprobe: w_B at the probe samples, per step of the segment
  void* work[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* lam[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* grad[3] = {nullptr, nullptr, nullptr};
  void* u0h[3] = {nullptr, nullptr, nullptr};   // initial physical H
  AdjCfg cfg[2];
  long long src_at = -1;
  double eps_src = 0;
  bool forward_done = false;
  double objective = 0;
  long long bytes = 0;
};

namespace {

void* arr_at(void* base, long long idx, const fdtd_t* h) {
  return (char*)base + (size_t)idx * (size_t)h->count * h->esize;
}

template <typename T>
fdtd::ProbeSet<T> probe_set(const fdtd_adj_t* a) {
  fdtd::ProbeSet<T> ps;
  ps.at = a->d_probe_at;
  ps.comp = a->d_probe_comp;
  ps.n = a->nprobe;
  return ps;
}

int copy_arrays(fdtd_t* h, void* const* dst, void* const* src, int first, int n) {
  for (int c = first; c < first + n; ++c)
    CK(cudaMemcpyAsync(dst[c], src[c], (size_t)h->count * h->esize, cudaMemcpyDeviceToDevice, h->stream));
  return FDTD_OK;
}

// One FADI step of the forward model on `st` (in place).  objective: add
// the step's probe energy to *d_acc.  rec_a, rec_b (recomputation): the
// per-node kernels also write each procedure's record D = E_in - E_out
// there, and w_B at the probe samples goes to wrec.
template <typename T>
int adj_forward_step(fdtd_adj_t* a, void* const* st, long long n, bool objective, void* const* rec_a,
                     void* const* rec_b, double* wrec) {
  fdtd_t* h = a->h;
  const double post_a = 0.5 * h->dt * source_value(h, n);
  const double post_b = 0.5 * h->dt * source_value(h, n + 1);
  auto proc = [&](int slot, void* const* rec) -> int {
    const ProcCoef& P = h->proc[slot];
    return fork_pairs(h, [&](int q) -> int {
      const PairGeom& g = h->geom[P.op][q];
      fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, st, st);
      if (rec) p.d_out = (T*)rec[g.ec];
      return launch_pair<T>(h, g, p);
    });
  };
  int rc = proc(0, rec_a);
  if (rc) return rc;
  if (h->src_comp >= 0 && (rc = add_point(h, st[h->src_comp], post_a))) return rc;
  const bool probes = a->nprobe && (objective || wrec);
  if (probes) {
    fdtd::probe_energy_kernel<T><<<1, 256, 0, h->stream>>>(probe_set<T>(a), (const T*)st[0], (const T*)st[1],
                                                           (const T*)st[2], a->d_stash, a->d_acc, 0, nullptr);
    CK(cudaGetLastError());
  }
  if ((rc = proc(1, rec_b))) return rc;
  if (probes) {
    fdtd::probe_energy_kernel<T><<<1, 256, 0, h->stream>>>(probe_set<T>(a), (const T*)st[0], (const T*)st[1],
                                                           (const T*)st[2], a->d_stash, a->d_acc,
                                                           objective ? 1 : 2, wrec);
    CK(cudaGetLastError());
  }
  if (h->src_comp >= 0 && (rc = add_point(h, st[h->src_comp], post_b))) return rc;
  return FDTD_OK;
}

// The three adjoint pair launches of procedure `slot` on lam (in place).
template <typename T>
int adj_procedure(fdtd_adj_t* a, int slot, void* const* rec, int only_axis = -1) {
  fdtd_t* h = a->h;
  const ProcCoef& P = h->proc[slot];
  auto pair = [&](int q) -> int {
    const PairGeom& g = h->geom[P.op][q];
    if (g.empty()) return FDTD_OK;
    if (only_axis >= 0 && (g.rows || (g.axis == AX_Y ? 0 : 1) != only_axis)) return FDTD_OK;
    fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, a->lam, a->lam);
    const T ks = p.ks, kd = p.kd;
    p.ks = -kd;  // transposed couplings
    p.kd = -ks;
    fdtd::AdjExtra<T> x;
    x.d = (const T*)rec[g.ec];
    x.grad = a->grad[g.ec];
    x.inv_h = 1.0 / P.h;
    h->launches++;
    if (g.rows) {
      switch (pick_rows_L(g.N)) {
        case 1: launch_adj_rows_L<T, 1>(h, g, p, x); break;
        case 2: launch_adj_rows_L<T, 2>(h, g, p, x); break;
        case 4: launch_adj_rows_L<T, 4>(h, g, p, x); break;
        case 8: launch_adj_rows_L<T, 8>(h, g, p, x); break;
        case 12: launch_adj_rows_L<T, 12>(h, g, p, x); break;
        case 16: launch_adj_rows_L<T, 16>(h, g, p, x); break;
        case 24: launch_adj_rows_L<T, 24>(h, g, p, x); break;
        case 32: launch_adj_rows_L<T, 32>(h, g, p, x); break;
        default: return FDTD_ERR_UNSUPPORTED;
      }
    } else {
      const AdjCfg& c = a->cfg[g.axis == AX_Y ? 0 : 1];
      if (!c.ok) return FDTD_ERR_UNSUPPORTED;
      if (c.lanes == 32 && c.L == 8) launch_adj_strided_L<T, 32, 8>(h, g, p, x);
      else if (c.lanes == 32 && c.L == 16) launch_adj_strided_L<T, 32, 16>(h, g, p, x);
      else if (c.lanes == 16 && c.L == 8) launch_adj_strided_L<T, 16, 8>(h, g, p, x);
      else if (c.lanes == 16 && c.L == 16) launch_adj_strided_L<T, 16, 16>(h, g, p, x);
      else if (c.lanes == 16 && c.L == 32) launch_adj_strided_L<T, 16, 32>(h, g, p, x);
      else if (c.lanes == 8 && c.L == 32) launch_adj_strided_L<T, 8, 32>(h, g, p, x);
      else return FDTD_ERR_UNSUPPORTED;
    }
    CK(cudaGetLastError());
    return FDTD_OK;
  };
  if (only_axis >= 0) {  // tuning: one direction, on the handle's stream
    for (int q = 0; q < 3; ++q)
      if (int rc = pair(q)) return rc;
    return FDTD_OK;
  }
  // the three transposed pairs write disjoint adjoint and gradient arrays
  return fork_pairs(h, pair);
}

template <typename T>
int adj_point_term(fdtd_adj_t* a, double post) {
  fdtd_t* h = a->h;
  if (h->src_comp < 0 || post == 0.0) return FDTD_OK;
  // post = (h/2) f with f proportional to 1/eps at the source sample
  fdtd::grad_point_kernel<T><<<1, 32, 0, h->stream>>>(a->grad[h->src_comp], (const T*)a->lam[h->src_comp],
                                                      a->src_at, -post / a->eps_src);
  CK(cudaGetLastError());
  return FDTD_OK;
}

template <typename T>
int adj_inject(fdtd_adj_t* a, const double* wrec, double jbar) {
  fdtd_t* h = a->h;
  if (!a->nprobe) return FDTD_OK;
  const unsigned blocks = (unsigned)std::min(1024, (a->nprobe + 255) / 256);
  fdtd::probe_inject_kernel<T><<<blocks, 256, 0, h->stream>>>(probe_set<T>(a), (T*)a->lam[0], (T*)a->lam[1],
                                                              (T*)a->lam[2], wrec, jbar);
  CK(cudaGetLastError());
  return FDTD_OK;
}

// Launch shape of the adjoint y/z kernels: every feasible candidate timed
// on the context's own (zeroed) adjoint arrays, both procedures.
template <typename T>
int adj_tune_t(fdtd_adj_t* a) {
  fdtd_t* h = a->h;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const std::string key = "adjoint|" + device_name() + "|p" + std::to_string(h->prec) + "|" +
                          std::to_string(h->nx) + "x" + std::to_string(h->ny) + "x" + std::to_string(h->nz);
  TuneVal v;
  if (tune_cache_get(key, &v) && adj_strided_fn<T>(v[0], v[1]) && adj_strided_fn<T>(v[2], v[3])) {
    a->cfg[0] = {true, v[0], v[1]};
    a->cfg[1] = {true, v[2], v[3]};
    return FDTD_OK;
  }
  const size_t bytes = (size_t)h->count * h->esize;
  for (int c = 0; c < 6; ++c) CK(cudaMemsetAsync(a->lam[c], 0, bytes, h->stream));
  for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(a->grad[c], 0, sizeof(double) * h->count, h->stream));
  static const int c32[][2] = {{32, 8}, {32, 16}, {16, 8}, {16, 16}, {16, 32}};
  static const int c64[][2] = {{16, 8}, {16, 16}, {16, 32}, {8, 32}, {16, 16}};
  const int(*cand)[2] = sizeof(T) == 8 ? c64 : c32;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int ax = 0; ax < 2; ++ax) {
    const int N = ax == 0 ? h->ny : h->nz;
    if (N < 2) continue;
    double best = -1;
    AdjCfg pick = a->cfg[ax];
    for (int q = 0; q < 5; ++q) {
      const int lanes = cand[q][0], L = cand[q][1];
      const int P = segments(N, L, lanes);
      cudaFuncAttributes fa;
      if (P > 32 || cudaFuncGetAttributes(&fa, adj_strided_fn<T>(lanes, L)) != cudaSuccess ||
          P * lanes > fa.maxThreadsPerBlock)
        continue;
      a->cfg[ax] = {true, lanes, L};
      double ms_best = 1e30;
      bool ok = true;
      for (int r = 0; r < 4 && ok; ++r) {
        cudaEventRecord(e0, h->stream);
        for (int slot = 0; slot < 2 && ok; ++slot)
          if (adj_procedure<T>(a, slot, h->f, ax) != FDTD_OK) ok = false;
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) ms_best = std::min(ms_best, (double)ms);
      }
      if (ok && (best < 0 || ms_best < best)) {
        best = ms_best;
        pick = a->cfg[ax];
      }
    }
    a->cfg[ax] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  tune_cache_put(key, {a->cfg[0].lanes, a->cfg[0].L, a->cfg[1].lanes, a->cfg[1].L, 0, 0});
  return FDTD_OK;
}

template <typename T>
int adj_forward_t(fdtd_adj_t* a) {
  fdtd_t* h = a->h;
  int rc;
  for (int c = 0; c < 3; ++c)
    CK(cudaMemcpyAsync(a->u0h[c], h->f[3 + c], (size_t)h->count * h->esize, cudaMemcpyDeviceToDevice, h->stream));
  if ((rc = scheme_init(h))) return rc;
  // launch shapes: forward (as fdtd_step would choose them) and adjoint
  if (!h->shape_tuned && h->desc.tune[0] == 0 && (rc = single_tune(h))) return rc;
  h->shape_tuned = true;
  if ((rc = adj_tune_t<T>(a))) return rc;
  CK(cudaMemsetAsync(a->d_acc, 0, sizeof(double), h->stream));
  for (long long n = 0; n < a->nsteps; ++n) {
    if (n % a->every == 0) {
      void* dst[6];
      for (int c = 0; c < 6; ++c) dst[c] = arr_at(a->ckpt, (n / a->every) * 6 + c, h);
      if ((rc = copy_arrays(h, dst, h->f, 0, 6))) return rc;
    }
    if ((rc = adj_forward_step<T>(a, h->f, n, true, nullptr, nullptr, nullptr))) return rc;
    h->steps++;
  }
  h->output_valid = false;
  CK(cudaMemcpyAsync(&a->objective, a->d_acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

template <typename T>
int adj_backward_t(fdtd_adj_t* a, double jbar) {
  fdtd_t* h = a->h;
  int rc;
  const size_t bytes = (size_t)h->count * h->esize;
  for (int c = 0; c < 6; ++c) CK(cudaMemsetAsync(a->lam[c], 0, bytes, h->stream));
  for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(a->grad[c], 0, sizeof(double) * h->count, h->stream));
  auto slot = [&](int s, void** out) {
    for (int c = 0; c < 3; ++c) out[c] = arr_at(a->tape, (long long)s * 3 + c, h);
  };
  for (int seg = a->nseg - 1; seg >= 0; --seg) {
    const long long n0 = (long long)seg * a->every;
    const long long n1 = std::min(n0 + a->every, a->nsteps);
    void* src[6];
    for (int c = 0; c < 6; ++c) src[c] = arr_at(a->ckpt, (long long)seg * 6 + c, h);
    if ((rc = copy_arrays(h, a->work, src, 0, 6))) return rc;
    for (long long n = n0; n < n1; ++n) {
      const int m = (int)(n - n0);
      void *ra[3], *rb[3];
      slot(2 * m, ra);
      slot(2 * m + 1, rb);
      if ((rc = adj_forward_step<T>(a, a->work, n, false, ra, rb, a->d_wrec + (size_t)m * a->nprobe))) return rc;
    }
    for (long long n = n1 - 1; n >= n0; --n) {
      const int m = (int)(n - n0);
      void *ra[3], *rb[3];
      slot(2 * m, ra);
      slot(2 * m + 1, rb);
      const double* wrec = a->d_wrec + (size_t)m * a->nprobe;
      const double post_a = 0.5 * h->dt * source_value(h, n);
      const double post_b = 0.5 * h->dt * source_value(h, n + 1);
      // B procedure of step n: the objective's w_B term enters w-bar; with
      // it added to the E adjoint before the transposed solve, the output
      // E-bar = q y - E-bar' needs it added back once more
      if ((rc = adj_point_term<T>(a, post_b))) return rc;
      if ((rc = adj_inject<T>(a, wrec, jbar))) return rc;
      if ((rc = adj_procedure<T>(a, 1, rb))) return rc;
      if ((rc = adj_inject<T>(a, wrec, jbar))) return rc;
      // A procedure of step n
      if ((rc = adj_point_term<T>(a, post_a))) return rc;
      if ((rc = adj_procedure<T>(a, 0, ra))) return rc;
    }
  }
  // input initialization v0 = u0 + (dt/2) B u0 + (dt/2) f
  if ((rc = adj_point_term<T>(a, 0.5 * h->dt * source_value(h, 0)))) return rc;
  const ProcCoef& P = h->proc[1];
  for (int q = 0; q < 3; ++q) {
    const PairGeom& g = h->geom[P.op][q];
    if (g.empty() || g.N < 2) continue;
    void* in[6] = {nullptr, nullptr, nullptr, a->u0h[0], a->u0h[1], a->u0h[2]};
    in[g.ec] = a->lam[g.ec];
    fdtd::PairParams<T> p = make_params<T>(h, g, P.pc[q], 1.0, 1.0, -1.0, 1.0, in, in);
    const double sgn = -1.0;  // B pairs
    const double coef = -0.5 * h->dt * sgn / (spacing(h, g.axis) * kEps0 * kEps0);
    const long long total = g.n_lines() * (g.N - 1);
    const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 32));
    fdtd::init_grad_kernel<T><<<blocks, 256, 0, h->stream>>>(p, g.rows ? 1 : 0, (const T*)a->lam[g.ec],
                                                             h->eps_node[g.ec], a->grad[g.ec], coef);
    CK(cudaGetLastError());
  }
  const long long cells = (long long)h->nx * h->ny * h->nz;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((cells + 255) / 256, 152LL * 32));
  fdtd::cell_grad_kernel<<<blocks, 256, 0, h->stream>>>(a->grad[0], a->grad[1], a->grad[2], h->nx, h->ny, h->nz,
                                                        h->pitch, h->plane, kEps0, a->d_cell);
  CK(cudaGetLastError());
  return FDTD_OK;
}

void adj_free(fdtd_adj_t* a) {
  void* ptrs[] = {a->d_probe_at, a->d_probe_comp, a->d_stash, a->d_acc, a->d_cell, a->ckpt, a->tape, a->d_wrec};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int c = 0; c < 6; ++c) {
    if (a->work[c]) cudaFree(a->work[c]);
    if (a->lam[c]) cudaFree(a->lam[c]);
  }
  for (int c = 0; c < 3; ++c) {
    if (a->grad[c]) cudaFree(a->grad[c]);
    if (a->u0h[c]) cudaFree(a->u0h[c]);
  }
}

}  // namespace

extern "C" {

int fdtd_adj_create(fdtd_t* h, const int32_t block[6], int64_t nsteps, int32_t checkpoint_every,
                    fdtd_adj_t** out) {
  if (!h || !block || !out || nsteps < 1 || checkpoint_every < 1) return FDTD_ERR_INVALID_ARG;
  *out = nullptr;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (h->scheme != FDTD_FADI || !h->per_node || h->mu_var || h->lossy || h->order != 2)
    return FDTD_ERR_UNSUPPORTED;
  if (!h->pending_init || h->steps != 0) return FDTD_ERR_STATE;
  if (h->nprobes > 0) return FDTD_ERR_UNSUPPORTED;
  const int i0 = block[0], i1 = block[1], j0 = block[2], j1 = block[3], k0 = block[4], k1 = block[5];
  if (i0 < 0 || j0 < 0 || k0 < 0 || i1 < i0 || j1 < j0 || k1 < k0 || i1 > h->nx + 1 || j1 > h->ny + 1 ||
      k1 > h->nz + 1)
    return FDTD_ERR_INVALID_ARG;
  fdtd_adj_t* a = new (std::nothrow) fdtd_adj_s();
  if (!a) return FDTD_ERR_OOM;
  a->h = h;
  a->nsteps = nsteps;
  a->every = checkpoint_every;
  a->nseg = (int)((nsteps + checkpoint_every - 1) / checkpoint_every);
  // probe samples: interior E samples whose index (i, j, k) lies in the block
  std::vector<long long> at;
  std::vector<int> comp;
  for (int c = 0; c < 3; ++c) {
    int sx, sy, sz;
    comp_extent(c, h->nx, h->ny, h->nz, &sx, &sy, &sz);
    for (int k = k0; k < std::min(k1, sz); ++k)
      for (int j = j0; j < std::min(j1, sy); ++j)
        for (int i = i0; i < std::min(i1, sx); ++i) {
          const bool wall_x = (c != EX) && (i == 0 || i == h->nx);
          const bool wall_y = (c != EY) && (j == 0 || j == h->ny);
          const bool wall_z = (c != EZ) && (k == 0 || k == h->nz);
          if (wall_x || wall_y || wall_z) continue;
          at.push_back(elem_index(h, i, j, k));
          comp.push_back(c);
        }
  }
  a->nprobe = (int)at.size();
  if (h->src_comp >= 0) {
    a->src_at = elem_index(h, h->src_i, h->src_j, h->src_k);
    double er = 1.0;
    if (cudaMemcpy(&er, h->eps_node[h->src_comp] + a->src_at, sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      delete a;
      return FDTD_ERR_CUDA;
    }
    a->eps_src = kEps0 * er;
  }
  const size_t arr = (size_t)h->count * h->esize;
  bool ok = true;
  auto alloc = [&](void** p, size_t n) {
    if (!ok) return;
    if (dev_malloc((void**)p, n) != cudaSuccess) ok = false;
    else a->bytes += (long long)n;
  };
  alloc((void**)&a->d_probe_at, sizeof(long long) * std::max<size_t>(1, at.size()));
  alloc((void**)&a->d_probe_comp, sizeof(int) * std::max<size_t>(1, comp.size()));
  alloc((void**)&a->d_stash, sizeof(double) * std::max<size_t>(1, at.size()));
  alloc((void**)&a->d_acc, sizeof(double));
  alloc((void**)&a->d_cell, sizeof(double) * (size_t)h->nx * h->ny * h->nz);
  alloc(&a->ckpt, arr * 6 * (size_t)a->nseg);
  alloc(&a->tape, arr * 3 * (size_t)(2 * checkpoint_every));
  alloc((void**)&a->d_wrec, sizeof(double) * std::max<size_t>(1, at.size()) * (size_t)checkpoint_every);
  for (int c = 0; c < 6; ++c) {
    alloc(&a->work[c], arr);
    alloc(&a->lam[c], arr);
  }
  for (int c = 0; c < 3; ++c) {
    alloc((void**)&a->grad[c], sizeof(double) * h->count);
    alloc(&a->u0h[c], arr);
  }
  if (!ok) {
    cudaGetLastError();
    adj_free(a);
    delete a;
    return FDTD_ERR_OOM;
  }
  if (!at.empty() &&
      (cudaMemcpy(a->d_probe_at, at.data(), sizeof(long long) * at.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(a->d_probe_comp, comp.data(), sizeof(int) * comp.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    adj_free(a);
    delete a;
    return FDTD_ERR_CUDA;
  }
  for (int ax = 0; ax < 2; ++ax) {
    const int N = ax == 0 ? h->ny : h->nz;
    a->cfg[ax] = h->prec == FDTD_F64 ? adj_strided_cfg<double>(N) : adj_strided_cfg<float>(N);
    if (!a->cfg[ax].ok && N >= 2) {
      adj_free(a);
      delete a;
      return FDTD_ERR_UNSUPPORTED;
    }
  }
  *out = a;
  return FDTD_OK;
}

int fdtd_adj_forward(fdtd_adj_t* a, double* objective) {
  if (!a || !objective) return FDTD_ERR_INVALID_ARG;
  fdtd_t* h = a->h;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (a->forward_done || !h->pending_init || h->steps != 0) return FDTD_ERR_STATE;
  NvtxScope range("adjoint forward");
  int rc = h->prec == FDTD_F64 ? adj_forward_t<double>(a) : adj_forward_t<float>(a);
  if (rc) return rc;
  a->forward_done = true;
  *objective = a->objective;
  return FDTD_OK;
}

int fdtd_adj_backward(fdtd_adj_t* a, double jbar, double* grad_eps_r, int on_device) {
  if (!a || !grad_eps_r || !std::isfinite(jbar)) return FDTD_ERR_INVALID_ARG;
  fdtd_t* h = a->h;
  if (h->poisoned) return FDTD_ERR_STATE;
  if (!a->forward_done) return FDTD_ERR_STATE;
  NvtxScope range("adjoint backward");
  int rc = h->prec == FDTD_F64 ? adj_backward_t<double>(a, jbar) : adj_backward_t<float>(a, jbar);
  if (rc) return rc;
  const size_t n = sizeof(double) * (size_t)h->nx * h->ny * h->nz;
  CK(cudaMemcpyAsync(grad_eps_r, a->d_cell, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

int fdtd_adj_memory(const fdtd_adj_t* a, int64_t* bytes) {
  if (!a || !bytes) return FDTD_ERR_INVALID_ARG;
  *bytes = a->bytes;
  return FDTD_OK;
}

int fdtd_adj_destroy(fdtd_adj_t* a) {
  if (!a) return FDTD_OK;
  cudaStreamSynchronize(a->h->stream);
  adj_free(a);
  delete a;
  return FDTD_OK;
}

}  // extern "C"
