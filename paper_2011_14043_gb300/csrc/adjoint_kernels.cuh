// Adjoint (reverse-mode) kernels of the FADI time stepper with per-node
// media, for gradients of a probe-energy objective with respect to eps.
//
// One forward procedure on a pair (Sec. III, Eqs. 37-44, rows scaled by
// q = 1/b into the symmetric form S = q T):
//     S w = q E + ks (H_j - H_{j-1});  H_f += kd (w_{f+1} - w_f);  E = w - E
// is linear in (E, H).  Its transpose, for adjoints (Ebar', Hbar') of the
// outputs, has the same shape with the couplings exchanged:
//     S y = Ebar' - kd (Hbar'_j - Hbar'_{j-1})
//     Hbar_f = Hbar'_f - ks (y_{f+1} - y_f)
//     Ebar   = q y - Ebar'
// (T^{-T} = diag(q) S^{-1} because S is symmetric), so the same pivots of S
// serve both directions.  The eps dependence of b = h/(2 eps) enters through
// the RHS term and T; both collapse to one local product,
//     dJ/d eps_j += (1/h) y_j D_j,   D_j = 2 E_j - w_j,
// with E the forward E state before the procedure and w its solve; D is
// what the forward kernels record (d_out = E_in - E_out, the subtraction
// of Eqs. 40/47 being E_out = w - E).  Derivation: b_j (s D_h H + 1/2 Lam w)_j
// = 1/2 w_j - E_j from the forward row, d b_j/d eps_j = -b_j/eps_j and
// q_j/eps_j = 2/h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "line_kernels.cuh"

namespace fdtd {

template <typename T>
struct AdjExtra {
  const T* d;         // forward record D = 2 E - w of this pair's component
  double* grad;       // dJ/d eps per E sample (field layout), accumulated
  double inv_h;       // 1 / procedure length
};

// Store of one adjoint node: H update, E output, eps gradient.
template <typename T, int L>
__device__ __forceinline__ void adj_store_node(const PairParams<T>& p, const AdjExtra<T>& x, long long at, int j,
                                               T E, T H, T q, T y, T ynext) {
  p.e_out[at] = fma(q, y, -E);
  p.h_out[at] = fma(p.kd, ynext - y, H);
  if (j >= 1) x.grad[at] += x.inv_h * (double)y * (double)x.d[at];
}

// Lines along y or z: the per-node strided solve with unit row scaling.
// p carries the exchanged couplings (p.ks = -kd, p.kd = -ks of the forward).
template <typename T, int LANES, int L>
__global__ void adj_strided_kernel(const PairParams<T> p, const AdjExtra<T> x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x % LANES;
  const int s = threadIdx.x / LANES;
  const int P = blockDim.x / LANES;
  const int i = blockIdx.x * LANES + lane;
  const int o = p.o_lo + blockIdx.y;
  const long long base = (long long)o * p.os + i;
  const bool active = (i >= p.lane_lo) && (i < p.lane_hi) && strided_line_ok(p, base);
  const int j0 = s * L;
  const int N = p.N;
  const long long ls = p.ls;

  T E[L], H[L], y[L], one[L], q[L], ibn[L], ibl[L];
  HiLo<T> ib_prev = {T(0), T(0)};
  T hm1 = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    one[t] = T(1);
    q[t] = T(0);
    ibn[t] = T(0);
    ibl[t] = T(0);
  }
  if (active) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        const long long at = base + (long long)j * ls;
        E[t] = p.e_in[at];
        H[t] = p.h_in[at];
        q[t] = p.nq[at];
        ibn[t] = p.nib[at];
        if constexpr (use_hilo<T>()) ibl[t] = p.nibl[at];
      }
    }
    if (j0 > 0 && j0 - 1 < N) {
      const long long at = base + (long long)(j0 - 1) * ls;
      hm1 = p.h_in[at];
      ib_prev.hi = p.nib[at];
      if constexpr (use_hilo<T>()) ib_prev.lo = p.nibl[at];
    }
  }
  T win;
  strided_solve<T, LANES, L, true>(p, j0, s, P, lane, sh, E, H, hm1, one, ibn, ibl, ib_prev, y, win);
  if (active) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        const T ynext = (t + 1 < L) ? y[t + 1] : win;
        adj_store_node<T, L>(p, x, base + (long long)j * ls, j, E[t], H[t], q[t], y[t], ynext);
      }
    }
  }
}

// x lines: one warp per line.
template <typename T, int L>
__global__ void adj_rows_kernel(const PairParams<T> p, const AdjExtra<T> x) {
  const unsigned FULL = 0xffffffffu;
  const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= (long long)p.n_o * p.n_o2) return;  // whole warp leaves together
  const int lane = threadIdx.x & 31;
  T E[L], H[L], q[L], ibn[L], ibl[L], one[L], y[L];
  row_load<T, L, true>(p, line, E, H, q, ibn, ibl);
#pragma unroll
  for (int t = 0; t < L; ++t) one[t] = T(1);
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const int j0 = lane * L;
  const int N = p.N;

  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1);
  if (lane == 0) hm1 = T(0);
  HiLo<T> ib_prev = {__shfl_up_sync(FULL, ibn[L - 1], 1), T(0)};
  if constexpr (use_hilo<T>()) ib_prev.lo = __shfl_up_sync(FULL, ibl[L - 1], 1);
  if (lane == 0) ib_prev = {T(0), T(0)};

  const HiLo<T> pf = phase_forward<T, L, 2>(p, j0, E, H, hm1, one, ibn, ibl, ib_prev, y);
  const T yin = warp_chain_forward<T>(y[L - 1], pf);
  const HiLo<T> pb = phase_backward<T, L, 2>(p, j0, yin, ibn, ibl, ib_prev, y);
  const T win = warp_chain_backward<T>(y[0], pb);
  phase_fix<T, L, 2>(p, j0, win, ibn, ibl, y);
  if (!row_ok<T, L>(p, base)) return;
  if (j0 + L <= N) {
    // whole segment: record, gradient and outputs as 16-byte vectors
    T dd[L];
    double g[L];
    load_seg<T, L>(x.d + base + j0, dd);
    load_seg<double, L>(x.grad + base + j0, g);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T ynext = (t + 1 < L) ? y[t + 1] : win;
      const T e_out = fma(q[t], y[t], -E[t]);
      H[t] = fma(p.kd, ynext - y[t], H[t]);
      E[t] = e_out;
      if (j0 + t >= 1) g[t] += x.inv_h * (double)y[t] * (double)dd[t];
    }
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
    store_seg<double, L>(x.grad + base + j0, g);
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        const T ynext = (t + 1 < L) ? y[t + 1] : win;
        adj_store_node<T, L>(p, x, base + j, j, E[t], H[t], q[t], y[t], ynext);
      }
    }
  }
}

// Probe samples of the objective J = sum_n sum_probe (w_B/2)^2.
template <typename T>
struct ProbeSet {
  const long long* at;   // sample offsets (field layout)
  const int* comp;       // E component of each sample (0..2)
  int n;
};

// mode 0 stashes the E state before the B procedure; mode 1 adds
// sum (w_B/2)^2 with w_B = E_after_B (before its source) + stash to *acc
// (forward pass); mode 2 writes w_B to wrec[k] (recomputation, for the
// reverse pass).
template <typename T>
__global__ void probe_energy_kernel(ProbeSet<T> ps, const T* e0, const T* e1, const T* e2, double* stash,
                                    double* acc, int mode, double* wrec) {
  const T* e[3] = {e0, e1, e2};
  double sum = 0.0;
  for (int k = threadIdx.x; k < ps.n; k += blockDim.x) {
    const double v = (double)e[ps.comp[k]][ps.at[k]];
    if (mode == 0) {
      stash[k] = v;
    } else if (mode == 1) {
      const double w = v + stash[k];
      sum += 0.25 * w * w;
    } else {
      wrec[k] = v + stash[k];
    }
  }
  if (mode != 1) return;
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) acc[0] += v;
  }
}

// Backward: lam_E += jbar * w_B/2 at the probe samples (w_B recorded by
// the recomputation).
template <typename T>
__global__ void probe_inject_kernel(ProbeSet<T> ps, T* l0, T* l1, T* l2, const double* wrec, double jbar) {
  T* lam[3] = {l0, l1, l2};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ps.n; k += gridDim.x * blockDim.x) {
    const int c = ps.comp[k];
    const long long at = ps.at[k];
    lam[c][at] = (T)((double)lam[c][at] + jbar * 0.5 * wrec[k]);
  }
}

// grad[at] += coef * lam[at] (the eps dependence of a point source).
template <typename T>
__global__ void grad_point_kernel(double* grad, const T* lam, long long at, double coef) {
  if (threadIdx.x == 0 && blockIdx.x == 0) grad[at] += coef * (double)lam[at];
}

// Input initialization v0 = u0 + (dt/2) B u0 (+ source): the E rows of B u0
// are sgn D_h H / eps, so dJ/d eps += lam0 * (-(dt/2) sgn D_h H / eps^2).
// p describes the B pair (geometry; p.h_in = the initial physical H).
template <typename T>
__global__ void init_grad_kernel(const PairParams<T> p, int rows, const T* lam, const double* eps_r, double* grad,
                                 double coef) {
  // coef = -(dt/2) * sgn / (d_eta * eps0)
  const long long n_lines = rows ? (long long)p.n_o * p.n_o2 : (long long)(p.lane_hi - p.lane_lo) * p.n_o;
  const long long total = n_lines * (p.N - 1);
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive x (as in explicit_pair_kernel)
    const int j = 1 + (rows ? (int)(g % (p.N - 1)) : (int)(g / n_lines));
    const long long line = rows ? g / (p.N - 1) : g % n_lines;
    long long base;
    if (rows) {
      const int jo = p.o_lo + (int)(line % p.n_o);
      const int ko = p.o2_lo + (int)(line / p.n_o);
      base = (long long)ko * p.os2 + (long long)jo * p.os;
    } else {
      const int nl = p.lane_hi - p.lane_lo;
      const int i = p.lane_lo + (int)(line % nl);
      const int o = p.o_lo + (int)(line / nl);
      base = (long long)o * p.os + i;
    }
    const long long at = base + (long long)j * p.ls;
    if (!FDTD_IN_RANGE(at - p.ls, at + 1, p.n_elem)) continue;
    const double er = eps_r[at];
    const double dh = (double)p.h_in[at] - (double)p.h_in[at - p.ls];
    grad[at] += coef * (double)lam[at] * dh / (er * er);
  }
}

// dJ/d eps_r per cell (compact [k][j][i] layout) from dJ/d eps per E sample:
// eps at an edge is eps0 times the mean over its in-domain cells, so each
// cell collects eps0 * g_sample / n_sample from its twelve edges.
__global__ void cell_grad_kernel(const double* gx, const double* gy, const double* gz, int nx, int ny, int nz,
                                 long long pitch, long long plane, double eps0, double* out) {
  const long long cells = (long long)nx * ny * nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / ((long long)nx * ny));
    // the samples read below lie between these two offsets
    if (!FDTD_IN_RANGE((long long)k * plane + (long long)j * pitch + i,
                       (long long)(k + 1) * plane + (long long)(j + 1) * pitch + i + 2, plane * (nz + 1)))
      continue;
    double acc = 0.0;
    // 1 / (in-domain cells along an axis next to node n): cells n-1 and n,
    // so the share of one sample is the product of two factors 1 or 1/2
    // (exact; no division)
    auto half = [](int n, int N) { return (n > 0 && n < N) ? 0.5 : 1.0; };
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj) {
        // Ex (i+1/2, j+dj, k+dk): cells (i, j+dj-1..j+dj, k+dk-1..k+dk)
        const long long at = (long long)(k + dk) * plane + (long long)(j + dj) * pitch + i;
        acc += gx[at] * (half(j + dj, ny) * half(k + dk, nz));
      }
    for (int dk = 0; dk < 2; ++dk)
      for (int di = 0; di < 2; ++di) {
        // Ey (i+di, j+1/2, k+dk)
        const long long at = (long long)(k + dk) * plane + (long long)j * pitch + i + di;
        acc += gy[at] * (half(i + di, nx) * half(k + dk, nz));
      }
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        // Ez (i+di, j+dj, k+1/2)
        const long long at = (long long)k * plane + (long long)(j + dj) * pitch + i + di;
        acc += gz[at] * (half(i + di, nx) * half(j + dj, ny));
      }
    out[c] = eps0 * acc;
  }
}

}  // namespace fdtd
