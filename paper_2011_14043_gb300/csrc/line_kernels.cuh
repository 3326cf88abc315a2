// Fused updating-procedure kernels (Sec. III) for one (E, H) component pair.
//
// For every grid line along the pair's axis the kernel performs, in one pass
// over HBM (each E and H sample read once and written once):
//   r_j = E_j + kb_j (H_j - H_{j-1})                  implicit RHS (Eqs. 38/41/45/48)
//   (1/2 - (b_j/2) d(d d)) w = r                       tridiagonal line solve
//   H_f <- H_f + kd (w_{f+1} - w_f)                    fused explicit update (Eqs. 43-44, 51-52)
//   E_j <- alpha w_j + beta E_j                        subtraction E <- w - E (Eqs. 40, 47, 50)
// Node j of a line and face j (between nodes j and j+1) sit at the same
// element offset of the E and H arrays.  Nodes 0 and N are PEC walls (w = 0).
//
// Line solve: the Thomas algorithm with factors precomputed in FP64 on the
// host (Sec. IV's "precomputed bidiagonally factorized elements"):
//   forward   y_j = r_j - m_j y_{j-1},       m_j = l_j / beta_{j-1}
//   backward  w_j = y_j / beta_j - c_j w_{j+1},  c_j = u_j / beta_j
// with 1/beta = 0 on wall nodes and beyond the line, which pins w = 0 there.
// Both recurrences are first-order linear, so a line is cut into segments:
// each thread runs the recurrences over its own segment from a zero carry,
// the segment carries are chained (a scan of affine maps x -> a + p x), and
// each thread adds carry * (product of its -m or -c) to its values.  This is
// exactly the sequential Thomas result, reassociated; nothing is stored
// outside registers and a few words of shared memory.
//
// Two layouts:
//   proc_strided_kernel  lines along y or z (stride pitch or plane).  LANES
//                        consecutive x lines form a coalesced row access;
//                        P = blockDim.x / LANES segments of L nodes each
//                        split every line; carries go through shared memory.
//   proc_rows_kernel     lines along x (contiguous).  One warp per line, lane
//                        l owns nodes/faces [l L, l L + L) loaded as 16-byte
//                        vectors; carries go through warp shuffles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

template <typename T>
struct PairParams {
  const T* e_in;
  const T* h_in;
  T* e_out;
  T* h_out;
  long long ls;        // element stride between consecutive nodes of a line
  long long os;        // strided: stride of the outer index; rows: stride of j
  long long os2;       // rows: stride of k
  int lane_lo, lane_hi;  // strided: active x range [lo, hi)
  int o_lo, n_o;         // strided: outer index range; rows: j range
  int o2_lo, n_o2;       // rows: k range
  int N;                 // cells along the line (nodes 0..N, faces 0..N-1)
  T kb;                  // uniform: RHS coupling s*b/d_eta
  T kd;                  // H update coupling s*d/d_eta
  T alpha, beta;         // E_out = alpha*w + beta*E_in
  const T* tab;          // uniform: [3][tlen] = 1/beta, m, c (zero beyond N and at walls)
  int tlen;
  const T* nkb;          // per-node: |b_j|/d_eta at each E node (field layout)
  const T* nib;          // per-node: 1/beta_j at each E node (field layout)
  T kb_sign;             // per-node: RHS coupling = kb_sign * nkb_j
  T dh;                  // per-node: off-diagonal o_j = -nkb_j * dh, dh = |d|/(2 d_eta)
  int src_i, src_o, src_o2, src_j;  // source node on this pair (-1: none)
  T src_rhs, src_post;   // added to r_j and to E_out at the source node
};

// ---------------------------------------------------------------------------
// Lines along y or z
// ---------------------------------------------------------------------------
template <typename T, int LANES, int L, bool PER_NODE>
__global__ void proc_strided_kernel(const PairParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);  // [4][P][LANES]
  const int lane = threadIdx.x % LANES;
  const int s = threadIdx.x / LANES;
  const int P = blockDim.x / LANES;
  const int i = blockIdx.x * LANES + lane;
  const int o = p.o_lo + blockIdx.y;
  const bool active = (i >= p.lane_lo) && (i < p.lane_hi);
  const long long base = (long long)o * p.os + i;
  const int j0 = s * L;
  const int N = p.N;
  const long long ls = p.ls;
  const bool src_line = (i == p.src_i) && (o == p.src_o);

  T E[L], H[L], y[L];
  T kbn[L];
  T ibn[L];
  T ib_prev = T(0);
  T hm1 = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    if (PER_NODE) { kbn[t] = T(0); ibn[t] = T(0); }
  }
  if (active) {
    const T* pe = p.e_in + base;
    const T* ph = p.h_in + base;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        E[t] = pe[(long long)j * ls];
        H[t] = ph[(long long)j * ls];
        if (PER_NODE) {
          kbn[t] = p.nkb[base + (long long)j * ls];
          ibn[t] = p.nib[base + (long long)j * ls];
        }
      }
    }
    if (j0 > 0 && j0 - 1 < N) {
      hm1 = ph[(long long)(j0 - 1) * ls];
      if (PER_NODE) ib_prev = p.nib[base + (long long)(j0 - 1) * ls];
    }
  }

  // coefficient accessors
  auto m_of = [&](int t) -> T {
    if (PER_NODE) return -kbn[t] * p.dh * (t == 0 ? ib_prev : ibn[t - 1]);
    return p.tab[p.tlen + j0 + t];
  };
  auto c_of = [&](int t) -> T {
    if (PER_NODE) return -kbn[t] * p.dh * ibn[t];
    return p.tab[2 * p.tlen + j0 + t];
  };
  auto ib_of = [&](int t) -> T {
    if (PER_NODE) return ibn[t];
    return p.tab[j0 + t];
  };

  // right-hand side and local forward sweep (zero carry-in)
  T pf = T(1);
  {
    T hprev = hm1;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T kb = PER_NODE ? p.kb_sign * kbn[t] : p.kb;
      T r = E[t] + kb * (H[t] - hprev);
      hprev = H[t];
      if (src_line && (j0 + t) == p.src_j) r += p.src_rhs;
      const T m = m_of(t);
      y[t] = (t == 0) ? r : r - m * y[t - 1];
      pf *= -m;
    }
  }
  sh[(0 * P + s) * LANES + lane] = y[L - 1];
  sh[(1 * P + s) * LANES + lane] = pf;
  __syncthreads();
  if (s == 0) {
    T c = T(0);
    for (int q = 0; q < P; ++q) {
      c = sh[(0 * P + q) * LANES + lane] + sh[(1 * P + q) * LANES + lane] * c;
      sh[(0 * P + q) * LANES + lane] = c;
    }
  }
  __syncthreads();
  const T yin = (s > 0) ? sh[(0 * P + s - 1) * LANES + lane] : T(0);
  {
    T q = T(1);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      q *= -m_of(t);
      y[t] += q * yin;
    }
  }
  // local backward sweep (zero carry-in from the right)
  T pb = T(1);
  {
    T wn = T(0);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      const T c = c_of(t);
      y[t] = y[t] * ib_of(t) - c * wn;
      wn = y[t];
      pb *= -c;
    }
  }
  sh[(2 * P + s) * LANES + lane] = y[0];
  sh[(3 * P + s) * LANES + lane] = pb;
  __syncthreads();
  if (s == 0) {
    T c = T(0);
    for (int q = P - 1; q >= 0; --q) {
      c = sh[(2 * P + q) * LANES + lane] + sh[(3 * P + q) * LANES + lane] * c;
      sh[(2 * P + q) * LANES + lane] = c;
    }
  }
  __syncthreads();
  const T win = (s + 1 < P) ? sh[(2 * P + s + 1) * LANES + lane] : T(0);
  {
    T q = T(1);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      q *= -c_of(t);
      y[t] += q * win;
    }
  }

  // explicit H update, subtraction, store
  if (active) {
    T* pe = p.e_out + base;
    T* ph = p.h_out + base;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        const T wnext = (t + 1 < L) ? y[t + 1] : win;
        const T hn = H[t] + p.kd * (wnext - y[t]);
        T en = p.alpha * y[t] + p.beta * E[t];
        if (src_line && j == p.src_j) en += p.src_post;
        pe[(long long)j * ls] = en;
        ph[(long long)j * ls] = hn;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Lines along x
// ---------------------------------------------------------------------------
template <typename T, int L>
__device__ __forceinline__ void load_seg(const T* __restrict__ src, T (&v)[L]) {
  constexpr int BYTES = L * (int)sizeof(T);
  if constexpr (BYTES % 16 == 0) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
    for (int q = 0; q < BYTES / 16; ++q) {
      uint4 x = s4[q];
      const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
      for (int u = 0; u < 16 / (int)sizeof(T); ++u) v[q * (16 / (int)sizeof(T)) + u] = xs[u];
    }
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) v[t] = src[t];
  }
}

template <typename T, int L>
__device__ __forceinline__ void store_seg(T* dst, const T (&v)[L]) {
  constexpr int BYTES = L * (int)sizeof(T);
  if constexpr (BYTES % 16 == 0) {
    uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int q = 0; q < BYTES / 16; ++q) {
      uint4 x;
      T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
      for (int u = 0; u < 16 / (int)sizeof(T); ++u) xs[u] = v[q * (16 / (int)sizeof(T)) + u];
      d4[q] = x;
    }
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) dst[t] = v[t];
  }
}

template <typename T, int L, bool PER_NODE>
__global__ void proc_rows_kernel(const PairParams<T> p) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  if (line >= (long long)p.n_o * p.n_o2) return;  // whole warp leaves together
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const int j0 = lane * L;
  const int N = p.N;
  const bool src_line = (jo == p.src_o) && (ko == p.src_o2);

  // Segments never run past the padded row (the row pitch is >= 32*L);
  // values at nodes/faces >= N are forced to zero.
  T E[L], H[L], y[L];
  T kbn[L];
  T ibn[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    kbn[t] = T(0);
    ibn[t] = T(0);
  }
  if (j0 < N) {  // lanes wholly past the line end touch no memory
    load_seg<T, L>(p.e_in + base + j0, E);
    load_seg<T, L>(p.h_in + base + j0, H);
    if constexpr (PER_NODE) {
      load_seg<T, L>(p.nkb + base + j0, kbn);
      load_seg<T, L>(p.nib + base + j0, ibn);
    }
  }
#pragma unroll
  for (int t = 0; t < L; ++t) {
    if (j0 + t >= N) {
      E[t] = T(0);
      H[t] = T(0);
      kbn[t] = T(0);
      ibn[t] = T(0);
    }
  }
  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1);
  if (lane == 0) hm1 = T(0);
  T ib_prev = T(0);
  if (PER_NODE) {
    ib_prev = __shfl_up_sync(FULL, ibn[L - 1], 1);
    if (lane == 0) ib_prev = T(0);
  }
  const T* tab = p.tab;
  auto m_of = [&](int t) -> T {
    if (PER_NODE) return -kbn[t] * p.dh * (t == 0 ? ib_prev : ibn[t - 1]);
    return tab[p.tlen + j0 + t];
  };
  auto c_of = [&](int t) -> T {
    if (PER_NODE) return -kbn[t] * p.dh * ibn[t];
    return tab[2 * p.tlen + j0 + t];
  };
  auto ib_of = [&](int t) -> T {
    if (PER_NODE) return ibn[t];
    return tab[j0 + t];
  };

  // RHS and local forward sweep
  T pf = T(1);
  {
    T hprev = hm1;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T kb = PER_NODE ? p.kb_sign * kbn[t] : p.kb;
      T r = E[t] + kb * (H[t] - hprev);
      hprev = H[t];
      if (src_line && (j0 + t) == p.src_j) r += p.src_rhs;
      const T m = m_of(t);
      y[t] = (t == 0) ? r : r - m * y[t - 1];
      pf *= -m;
    }
  }
  // inclusive scan over lanes of x -> a + p x (Kogge-Stone)
  T a = y[L - 1], pp = pf;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T a_up = __shfl_up_sync(FULL, a, d);
    const T p_up = __shfl_up_sync(FULL, pp, d);
    if (lane >= d) {
      a = a + pp * a_up;
      pp = pp * p_up;
    }
  }
  T yin = __shfl_up_sync(FULL, a, 1);
  if (lane == 0) yin = T(0);
  {
    T q = T(1);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      q *= -m_of(t);
      y[t] += q * yin;
    }
  }
  // local backward sweep
  T pb = T(1);
  {
    T wn = T(0);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      const T c = c_of(t);
      y[t] = y[t] * ib_of(t) - c * wn;
      wn = y[t];
      pb *= -c;
    }
  }
  T b = y[0], qq = pb;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T b_dn = __shfl_down_sync(FULL, b, d);
    const T q_dn = __shfl_down_sync(FULL, qq, d);
    if (lane + d < 32) {
      b = b + qq * b_dn;
      qq = qq * q_dn;
    }
  }
  T win = __shfl_down_sync(FULL, b, 1);
  if (lane == 31) win = T(0);
  {
    T q = T(1);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      q *= -c_of(t);
      y[t] += q * win;
    }
  }
  // H update, subtraction, store (values beyond N are exactly zero)
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T wnext = (t + 1 < L) ? y[t + 1] : win;
    H[t] = H[t] + p.kd * (wnext - y[t]);
    T en = p.alpha * y[t] + p.beta * E[t];
    if (src_line && (j0 + t) == p.src_j) en += p.src_post;
    E[t] = en;
  }
  if (j0 + L <= N) {
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t < N) {
        p.e_out[base + j0 + t] = E[t];
        p.h_out[base + j0 + t] = H[t];
      }
    }
  }
}

}  // namespace fdtd
