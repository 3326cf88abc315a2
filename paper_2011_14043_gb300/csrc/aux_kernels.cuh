// Auxiliary kernels: explicit operator half-steps (FADI input
// initialization, Eq. 10), probe recording, FP64 energy reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "line_kernels.cuh"

namespace fdtd {

// Out-of-place explicit half-step of one pair of an operator O:
//   E_out_j = E_j + kb_j (H_j - H_{j-1})   at the interior nodes j = 1..N-1
//   H_out_f = H_f + kd (E_{f+1} - E_f)     at the faces f = 0..N-1
// on the pair's active lines (the same geometry as the procedure kernels).
// With kb = s*tau/(eps d_eta), kd = s*tau/(mu d_eta) this is (I + tau O).
template <typename T, bool PER_NODE>
__global__ void explicit_pair_kernel(const PairParams<T> p, int rows) {
  const long long n_lines = rows ? (long long)p.n_o * p.n_o2 : (long long)(p.lane_hi - p.lane_lo) * p.n_o;
  const long long total = n_lines * p.N;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    // consecutive threads take consecutive x: nodes of an x line, or the
    // same node of neighbouring y/z lines
    const int j = rows ? (int)(g % p.N) : (int)(g / n_lines);
    const long long line = rows ? g / p.N : g % n_lines;
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
    if (!FDTD_IN_RANGE(at - (j >= 1 ? p.ls : 0), at + (j + 1 < p.N ? p.ls : 0) + 1, p.n_elem)) continue;
    const T hf = p.h_in[at];
    if (j >= 1) {
      const T kb = PER_NODE ? p.ks / p.nq[at] : p.kb;   // s b_j / d_eta (h > 0)
      p.e_out[at] = p.e_in[at] + kb * (hf - p.h_in[at - p.ls]);
    } else {
      p.e_out[at] = p.e_in[at];
    }
    const T enext = (j + 1 < p.N) ? p.e_in[at + p.ls] : T(0);
    const T kd = p.nkd ? p.kd_scale * p.nkd[at] : p.kd;  // per-node mu: the face's coupling
    p.h_out[at] = hf + kd * (enext - p.e_in[at]);
  }
}

// y[i] += a * x[i] at one element (point source added to a state array).
template <typename T>
__global__ void add_point_kernel(T* y, long long at, double a) {
  if (threadIdx.x == 0 && blockIdx.x == 0) y[at] = (T)((double)y[at] + a);
}

// Loss part of the FADI input initialization (I + dt/2 B) u^0 in a lossy
// medium: out -= k (sigma / eps_r) in with k = dt / (4 eps0), sigma and eps_r
// per E node (device FP64, field layout) or uniform (null pointer).
template <typename T>
__global__ void loss_scale_kernel(T* __restrict__ out, const T* __restrict__ in, const double* __restrict__ sig,
                                  const double* __restrict__ epsr, double sig_u, double eps_u, double k, long long n) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
    const double sg = sig ? sig[g] : sig_u;
    const double er = epsr ? epsr[g] : eps_u;
    // row padding holds eps_r = 0 and sigma = 0: leave it untouched
    if (sg > 0.0 && er > 0.0) out[g] = (T)((double)out[g] - k * sg / er * (double)in[g]);
  }
}

// y[at] += coef * table[*step + offset] (0 outside the table): a point
// source whose value is read on the device, so that steps replayed from one
// captured graph see each step's value.  The product is rounded before the
// add (no fused multiply-add), as when the host forms coef * f.
template <typename T>
__global__ void add_point_table_kernel(T* y, long long at, const double* table, long long len,
                                       const long long* step, int offset, double coef) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const long long n = *step + offset;
    const double v = (n >= 0 && n < len) ? table[n] : 0.0;
    y[at] = (T)__dadd_rn((double)y[at], __dmul_rn(coef, v));
  }
}

// mode 0: *step = value;  mode 1: *step += 1.
__global__ void step_counter_kernel(long long* step, long long value, int mode) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step = mode == 0 ? value : *step + 1;
}

// Compact [sz][sy][sx] <-> padded (plane, pitch) layout of one component,
// for host copies staged through a contiguous device buffer: one row (fixed
// j, k) per block iteration, threads along x (no per-element division).
template <typename T>
__global__ void unpack_kernel(const T* __restrict__ src, T* __restrict__ dst, int sx, int sy, int sz,
                              long long pitch, long long plane) {
  const long long rows = (long long)sy * sz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long long at = (r / sy) * plane + (r % sy) * pitch;
    if (!FDTD_IN_RANGE(at, at + sx, (long long)sz * plane)) continue;
    for (int i = threadIdx.x; i < sx; i += blockDim.x) dst[at + i] = src[r * sx + i];
  }
}

template <typename T>
__global__ void pack_kernel(const T* __restrict__ src, T* __restrict__ dst, int sx, int sy, int sz, long long pitch,
                            long long plane) {
  const long long rows = (long long)sy * sz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long long at = (r / sy) * plane + (r % sy) * pitch;
    if (!FDTD_IN_RANGE(at, at + sx, (long long)sz * plane)) continue;
    for (int i = threadIdx.x; i < sx; i += blockDim.x) dst[r * sx + i] = src[at + i];
  }
}

// Zero the tangential E of component comp (0..2: Ex, Ey, Ez) on the PEC
// walls: whole rows on the y or z walls, the two end samples i = 0 and
// i = nx of the other rows for Ey and Ez (walls normal to x).
template <typename T>
__global__ void zero_walls_kernel(T* e, int comp, int nx, int ny, int nz, long long pitch, long long plane) {
  int sx, sy, sz;
  if (comp == 0) { sx = nx; sy = ny + 1; sz = nz + 1; }
  else if (comp == 1) { sx = nx + 1; sy = ny; sz = nz + 1; }
  else { sx = nx + 1; sy = ny + 1; sz = nz; }
  const long long rows = (long long)sy * sz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = (int)(r % sy);
    const int k = (int)(r / sy);
    const long long at = (long long)k * plane + (long long)j * pitch;
    if (!FDTD_IN_RANGE(at, at + sx, plane * (nz + 1))) continue;
    bool whole;
    if (comp == 0) whole = (j == 0 || j == ny || k == 0 || k == nz);
    else if (comp == 1) whole = (k == 0 || k == nz);
    else whole = (j == 0 || j == ny);
    if (whole) {
      for (int i = threadIdx.x; i < sx; i += blockDim.x) e[at + i] = T(0);
    } else if (comp != 0 && threadIdx.x == 0) {
      e[at] = T(0);
      e[at + nx] = T(0);
    }
  }
}

constexpr int kMaxProbes = 16;

template <typename T>
struct ProbeParams {
  const T* arr[kMaxProbes];
  long long at[kMaxProbes];
  double sub[kMaxProbes];  // mode 1: subtracted from value (a source added after the solve)
  int n;
};

// mode 0: stash[p] = value;  mode 1: out[p][col] = (stash[p] + value - sub[p])/2;
// mode 2: out[p][col] = value.
template <typename T>
__global__ void probe_kernel(const ProbeParams<T> pp, double* stash, double* out, long long ld,
                             long long col, int mode) {
  const int q = threadIdx.x;
  if (q >= pp.n) return;
  const double v = (double)pp.arr[q][pp.at[q]];
  if (mode == 0) {
    stash[q] = v;
  } else if (mode == 1) {
    out[(long long)q * ld + col] = 0.5 * (stash[q] + v - pp.sub[q]);
  } else {
    out[(long long)q * ld + col] = v;
  }
}

// The six components' weighted sums of squares in one launch: per block one
// FP64 partial sum of w_c * (wv[g]) * x_c[g]^2 over the concatenated arrays
// (each n elements, n a multiple of 4, 16-byte aligned), read as 16-byte
// vectors.  FP32 fields with scalar weights sum the 4 squares of a vector in
// FP32 (FMA) before the FP64 accumulation: one FP64 operation per 4
// elements, so the reduction runs at memory speed instead of at the FP64
// rate; the rounding of that 4-term sum is 2^-22 relative, far below the
// FP32 values' own.  Everything else accumulates each element in FP64.
struct Energy6 {
  const void* x[6];
  const double* wv[6];
  double w[6];
};

template <typename T>
__global__ void weighted_sumsq6_kernel(const Energy6 a, long long n, double* partial) {
  const long long n4 = n / 4;
  double acc = 0.0;
  for (int c = 0; c < 6; ++c) {
    const double w = a.w[c];
    const double* wv = a.wv[c];
    double ac = 0.0;
    if constexpr (sizeof(T) == 4) {
      const float4* x4 = reinterpret_cast<const float4*>(a.x[c]);
      for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n4;
           g += (long long)gridDim.x * blockDim.x) {
        const float4 v = x4[g];
        if (wv) {
          ac += wv[4 * g] * ((double)v.x * v.x) + wv[4 * g + 1] * ((double)v.y * v.y) +
                wv[4 * g + 2] * ((double)v.z * v.z) + wv[4 * g + 3] * ((double)v.w * v.w);
        } else {
          ac += (double)fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
        }
      }
    } else {
      const double2* x2 = reinterpret_cast<const double2*>(a.x[c]);
      for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n / 2;
           g += (long long)gridDim.x * blockDim.x) {
        const double2 v = x2[g];
        ac += (wv ? wv[2 * g] : 1.0) * v.x * v.x + (wv ? wv[2 * g + 1] : 1.0) * v.y * v.y;
      }
    }
    acc += w * ac;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

// FP64 FMA throughput probe: every thread runs 8 independent chains of
// `iters` FMAs x <- x a + b (|a| < 1, so the values stay bounded); the sum is
// stored only under a condition the host makes false, which keeps the work
// from being optimised away.
__global__ void fp64_fma_probe_kernel(double* out, long long iters, double a, double b, double never) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double sum = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) sum += x[c];
  if (sum == never) out[0] = sum;
}

}  // namespace fdtd
