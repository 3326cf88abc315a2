// Fourth-order difference operators (the higher-order variant of the
// updating procedure).
//
// The paper names higher-order difference operators as one of the variants
// its fundamental schemes leave room for (end of Sec. III-A), without
// formulae.  Here every first difference of the procedure is the
// fourth-order staggered central difference
//     (c1 (u_{+1/2} - u_{-1/2}) + c2 (u_{+3/2} - u_{-3/2})) / d,  c1 = 9/8, c2 = -1/24,
// and the points past a PEC wall are images: tangential E is odd about the
// wall, the H samples half a cell off it are even.  The two differences are
// then exact negative transposes of each other (A and B stay skew in the
// energy product), and eliminating H gives line systems of bandwidth 3:
//     1/2 w - (b/2) D(d D w) = E + s b D H,   H += s d D w,   E <- w - E.
// proc_line4_tile_kernel (FP32 fields, lines of at most 512 cells) gives a
// block of 256 threads 32 lines: all threads stage the lines' H in shared
// memory and keep their E values in registers, form the right-hand
// sides in a shared line buffer, one warp runs the forward and backward
// sweeps of the banded LU in that buffer (one lane per line), and all
// threads write the H and E updates.  Every field value crosses HBM once
// each way.  proc_line4_kernel (one thread per line, the intermediate values
// in a field-shaped scratch array) takes longer lines and the explicit
// operator of the FADI initialization.
#pragma once

namespace fdtd {

// Banded LU factor rows (hi, lo) of one pair's line system, indexed by the
// node j = 1..N-1: L multipliers l1..l3 (unit diagonal), 1/u0 and u1..u3.
enum { T4_L1H = 0, T4_L1L, T4_L2H, T4_L2L, T4_L3H, T4_L3L, T4_IUH, T4_IUL, T4_U1H, T4_U1L, T4_U2H, T4_U2L,
       T4_U3H, T4_U3L, T4_ROWS };

// mode 0: the procedure (in place or not); mode 1: the explicit operator
// (I + tau O) of the pair, out of place (the FADI input initialization).
template <typename T>
__global__ void proc_line4_kernel(const PairParams<T> p, int rows, int mode) {
  const long long n_lines = rows ? (long long)p.n_o * p.n_o2 : (long long)(p.lane_hi - p.lane_lo) * p.n_o;
  const int N = p.N;
  const long long ls = p.ls;
  const T c1 = T(1.125);
  const T c2 = p.c2_4;
  for (long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x; line < n_lines;
       line += (long long)gridDim.x * blockDim.x) {
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
    if (!FDTD_IN_RANGE(base, base + (long long)N * ls + 1, p.n_elem)) continue;
    const T* E = p.e_in + base;
    const T* H = p.h_in + base;
    // H at face f with even images; E at node m with odd images (walls 0)
    auto hface = [&](int f) -> T {
      const int g = f < 0 ? -1 - f : (f > N - 1 ? 2 * N - 1 - f : f);
      return H[(long long)g * ls];
    };
    auto enode = [&](const T* a, int m) -> T {
      if (m <= 0 || m >= N) {
        if (m < 0 && -m < N) return -a[(long long)(-m) * ls];
        if (m > N && 2 * N - m > 0) return -a[(long long)(2 * N - m) * ls];
        return T(0);
      }
      return a[(long long)m * ls];
    };
    T* Eo = p.e_out + base;
    T* Ho = p.h_out + base;
    if (mode == 1) {
      // (I + tau O): E += kb D H at the interior nodes, H += kd D E at the faces
      for (int f = 0; f < N; ++f) {
        const T de = c1 * (enode(E, f + 1) - enode(E, f)) + c2 * (enode(E, f + 2) - enode(E, f - 1));
        Ho[(long long)f * ls] = H[(long long)f * ls] + p.kd * de;
      }
      for (int j = 0; j < N; ++j) {
        T v = E[(long long)j * ls];
        if (j >= 1) v += p.kb * (c1 * (hface(j) - hface(j - 1)) + c2 * (hface(j + 1) - hface(j - 2)));
        Eo[(long long)j * ls] = v;
      }
      continue;
    }
    T* W = p.tmp4 + base;
    auto tab = [&](int row_hi, int j) -> HiLo<T> {  // (hi, lo) of a factor row
      return {p.tab[row_hi * p.tlen + j], p.tab[(row_hi + 1) * p.tlen + j]};
    };
    // forward sweep of the banded LU, right-hand side on the fly
    T y1 = T(0), y2 = T(0), y3 = T(0);
    for (int j = 1; j <= N - 1; ++j) {
      const T dh = c1 * (hface(j) - hface(j - 1)) + c2 * (hface(j + 1) - hface(j - 2));
      const T r = fma(p.kb, dh, E[(long long)j * ls]);
      const HiLo<T> l1 = tab(T4_L1H, j), l2 = tab(T4_L2H, j), l3 = tab(T4_L3H, j);
      const T y = fma2(HiLo<T>{-l1.hi, -l1.lo}, y1, fma2(HiLo<T>{-l2.hi, -l2.lo}, y2,
                                                         fma2(HiLo<T>{-l3.hi, -l3.lo}, y3, r)));
      W[(long long)j * ls] = y;
      y3 = y2;
      y2 = y1;
      y1 = y;
    }
    // backward sweep
    T w1 = T(0), w2 = T(0), w3 = T(0);
    for (int j = N - 1; j >= 1; --j) {
      const HiLo<T> u1 = tab(T4_U1H, j), u2 = tab(T4_U2H, j), u3 = tab(T4_U3H, j);
      const HiLo<T> iu = tab(T4_IUH, j);
      const T t = fma2(HiLo<T>{-u1.hi, -u1.lo}, w1, fma2(HiLo<T>{-u2.hi, -u2.lo}, w2,
                                                         fma2(HiLo<T>{-u3.hi, -u3.lo}, w3, W[(long long)j * ls])));
      T w;
      if constexpr (use_hilo<T>()) w = fma(iu.hi, t, iu.lo * t);
      else w = iu.hi * t;
      W[(long long)j * ls] = w;
      w3 = w2;
      w2 = w1;
      w1 = w;
    }
    // explicit H update from w (faces), then the E update (nodes)
    for (int f = 0; f < N; ++f) {
      const T dw = c1 * (enode(W, f + 1) - enode(W, f)) + c2 * (enode(W, f + 2) - enode(W, f - 1));
      Ho[(long long)f * ls] = fma(p.kd, dw, H[(long long)f * ls]);
    }
    for (int j = 0; j < N; ++j) {
      const T w = (j >= 1) ? W[(long long)j * ls] : T(0);
      Eo[(long long)j * ls] = fma(p.alpha, w, p.beta * E[(long long)j * ls]);
    }
  }
}

// Lines of one block: LN = 32 (FP32) or 16 (FP64), 256 threads.  Lines along
// y and z are LN consecutive x at one outer index (tile x0 a multiple of LN,
// so every row of the tile starts on a 16-byte boundary and is read and
// written with 16-byte vectors); lines along x are LN consecutive rows.
template <typename T>
__host__ __device__ constexpr int line4_tile_lines() {
  return sizeof(T) == 4 ? 32 : 16;
}

// chunks of 32 nodes per line of the tiled kernel (N <= 32 CH)
__host__ __device__ constexpr int line4_tile_ch(int N) { return N <= 64 ? 2 : (N <= 256 ? 8 : 16); }

template <typename T>
__host__ __device__ constexpr int line4_tile_stride(bool rows) {
  // rows are stored transposed (node-major): one padding column keeps the
  // transposing stores of a warp on distinct banks
  return line4_tile_lines<T>() + (rows ? 1 : 0);
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

__device__ __forceinline__ float4 vec16_make(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 vec16_make(const double* a) { return make_double2(a[0], a[1]); }
__device__ __forceinline__ void vec16_split(float4 v, float* a) {
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}
__device__ __forceinline__ void vec16_split(double2 v, double* a) {
  a[0] = v.x;
  a[1] = v.y;
}

// CH chunks of 32 nodes per line (N <= 32 CH); the procedure only (mode 0).
template <typename T, bool ROWS, int CH>
__global__ void __launch_bounds__(256, (CH <= 8 ? 3 : 1)) proc_line4_tile_kernel(const PairParams<T> p) {
  constexpr int LN = line4_tile_lines<T>();
  constexpr int V = LN / 8;  // values of one thread in one chunk
  constexpr int S = line4_tile_stride<T>(ROWS);
  using VT = typename Vec16<T>::type;
  static_assert(sizeof(VT) == V * sizeof(T), "one 16-byte vector per chunk");
  extern __shared__ __align__(16) unsigned char smem4[];
  __shared__ long long s_base[LN];
  __shared__ int s_ok[LN];
  const int N = p.N;
  const long long ls = p.ls;
  T* sH = reinterpret_cast<T*>(smem4);  // faces 0..N-1 of the lines' H, [face][line]
  T* sW = sH + (size_t)N * S;           // nodes 1..N-1: right-hand side, then y, then w
  const int t = threadIdx.x;
  if (t < LN) {
    long long base = 0;
    bool ok = false;
    if constexpr (ROWS) {
      const long long line = (long long)blockIdx.x * LN + t;
      if (line < (long long)p.n_o * p.n_o2) {
        const int jo = p.o_lo + (int)(line % p.n_o);
        const int ko = p.o2_lo + (int)(line / p.n_o);
        base = (long long)ko * p.os2 + (long long)jo * p.os;
        ok = true;
      }
    } else {
      const int tiles = (p.lane_hi + LN - 1) / LN;
      const int i = (int)(blockIdx.x % tiles) * LN + t;
      const int o = p.o_lo + (int)(blockIdx.x / tiles);
      base = (long long)o * p.os + i;  // inactive lanes too: they sit in the vectors
      ok = i >= p.lane_lo && i < p.lane_hi;
    }
    ok = ok && FDTD_IN_RANGE(base, base + (long long)(N - 1) * ls + 1, p.n_elem);
    s_base[t] = base;
    s_ok[t] = ok ? 1 : 0;
  }
  __syncthreads();
  // value v of chunk c of this thread is node 32 c + jo of line lv(v)
  const int jo = ROWS ? (t & 31) : (t >> 3);
  auto lv = [&](int v) { return ROWS ? (t >> 5) + 8 * v : V * (t & 7) + v; };
  bool any_ok = false, all_ok = true;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    any_ok |= s_ok[lv(v)] != 0;
    all_ok &= s_ok[lv(v)] != 0;
  }
  // 1. H of the lines to shared memory, E to registers (one read of each)
  T Ev[CH][V];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 32 * c + jo;
#pragma unroll
    for (int v = 0; v < V; ++v) Ev[c][v] = T(0);
    if (j >= N) continue;
    if constexpr (!ROWS) {
      if (any_ok) {
        const long long at = s_base[lv(0)] + (long long)j * ls;
        VT hv = {}, ev = {};
        if (FDTD_IN_RANGE(at, at + V, p.n_elem)) {
          hv = *reinterpret_cast<const VT*>(p.h_in + at);
          ev = *reinterpret_cast<const VT*>(p.e_in + at);
        }
        *reinterpret_cast<VT*>(sH + (size_t)j * S + lv(0)) = hv;
        vec16_split(ev, Ev[c]);
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) sH[(size_t)j * S + lv(v)] = T(0);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int l = lv(v);
        T hv = T(0);
        if (s_ok[l]) {
          const long long at = s_base[l] + j;
          hv = p.h_in[at];
          Ev[c][v] = p.e_in[at];
        }
        sH[(size_t)j * S + l] = hv;
      }
    }
  }
  __syncthreads();
  const T c1 = T(1.125);
  const T c2 = p.c2_4;
  // H at face f (-2 <= f <= N) with even images about the walls
  auto hface = [&](int f, int l) -> T {
    const int g = f < 0 ? -1 - f : (f > N - 1 ? 2 * N - 1 - f : f);
    return sH[(size_t)g * S + l];
  };
  // y/z tiles: the V lanes of one thread are one 16-byte vector of a shared
  // row (rows of LN elements; a warp touches four whole rows)
  auto ldrow = [&](const T* a, int row, T* out) {
    vec16_split(*reinterpret_cast<const VT*>(a + (size_t)row * S + lv(0)), out);
  };
  // 2. right-hand sides r_j = E_j + kb D H at the interior nodes
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 32 * c + jo;
    if (j < 1 || j >= N) continue;
    if constexpr (!ROWS) {
      auto fimg = [&](int f) { return f < 0 ? -1 - f : (f > N - 1 ? 2 * N - 1 - f : f); };
      T h0[V], hm[V], hp[V], hm2[V], r[V];
      ldrow(sH, j, h0);
      ldrow(sH, fimg(j - 1), hm);
      ldrow(sH, fimg(j + 1), hp);
      ldrow(sH, fimg(j - 2), hm2);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T dh = c1 * (h0[v] - hm[v]) + c2 * (hp[v] - hm2[v]);
        r[v] = fma(p.kb, dh, Ev[c][v]);
      }
      *reinterpret_cast<VT*>(sW + (size_t)j * S + lv(0)) = vec16_make(r);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int l = lv(v);
        const T dh = c1 * (hface(j, l) - hface(j - 1, l)) + c2 * (hface(j + 1, l) - hface(j - 2, l));
        sW[(size_t)j * S + l] = fma(p.kb, dh, Ev[c][v]);
      }
    }
  }
  __syncthreads();
  // 3. The banded LU sweeps, one lane of warp 0 per line.  Nodes jc4..je4
  // take the converged factor rows from registers, in chunks of 8 whose
  // shared-memory operands are loaded one chunk ahead; the nodes near the
  // walls read the table.  The arithmetic is the same as with the table
  // everywhere.
  if (t < LN) {
    T* w_l = sW + t;
    auto tab = [&](int row_hi, int j) -> HiLo<T> {
      return {__ldg(p.tab + row_hi * p.tlen + j), __ldg(p.tab + (row_hi + 1) * p.tlen + j)};
    };
    auto neg = [](HiLo<T> a) -> HiLo<T> { return {-a.hi, -a.lo}; };
    const int ja = min(max(p.jc4, 1), N);       // table nodes [1, ja)
    const int jb = max(ja, min(p.je4 + 1, N));  // converged nodes [ja, jb); table [jb, N)
    T y1 = T(0), y2 = T(0), y3 = T(0);
    auto fstep = [&](int j, HiLo<T> a1, HiLo<T> a2, HiLo<T> a3, T r) {
      const T y = fma2(neg(a1), y1, fma2(neg(a2), y2, fma2(neg(a3), y3, r)));
      w_l[(size_t)j * S] = y;
      y3 = y2;
      y2 = y1;
      y1 = y;
    };
    int j = 1;
    for (; j < ja; ++j) fstep(j, tab(T4_L1H, j), tab(T4_L2H, j), tab(T4_L3H, j), w_l[(size_t)j * S]);
    {
      const HiLo<T> k1 = {p.cv4[T4_L1H], p.cv4[T4_L1L]}, k2 = {p.cv4[T4_L2H], p.cv4[T4_L2L]},
                    k3 = {p.cv4[T4_L3H], p.cv4[T4_L3L]};
      T rn[8];
      if (j + 8 <= jb) {
#pragma unroll
        for (int u = 0; u < 8; ++u) rn[u] = w_l[(size_t)(j + u) * S];
      }
      for (; j + 8 <= jb; j += 8) {
        T r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = rn[u];
        if (j + 16 <= jb) {
#pragma unroll
          for (int u = 0; u < 8; ++u) rn[u] = w_l[(size_t)(j + 8 + u) * S];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) fstep(j + u, k1, k2, k3, r[u]);
      }
      for (; j < jb; ++j) fstep(j, k1, k2, k3, w_l[(size_t)j * S]);
    }
    for (; j <= N - 1; ++j) fstep(j, tab(T4_L1H, j), tab(T4_L2H, j), tab(T4_L3H, j), w_l[(size_t)j * S]);
    T w1 = T(0), w2 = T(0), w3 = T(0);
    auto bstep = [&](int j, HiLo<T> a1, HiLo<T> a2, HiLo<T> a3, HiLo<T> iu, T yv) {
      const T tt = fma2(neg(a1), w1, fma2(neg(a2), w2, fma2(neg(a3), w3, yv)));
      T w;
      if constexpr (use_hilo<T>()) w = fma(iu.hi, tt, iu.lo * tt);
      else w = iu.hi * tt;
      w_l[(size_t)j * S] = w;
      w3 = w2;
      w2 = w1;
      w1 = w;
    };
    j = N - 1;
    for (; j >= jb; --j)
      bstep(j, tab(T4_U1H, j), tab(T4_U2H, j), tab(T4_U3H, j), tab(T4_IUH, j), w_l[(size_t)j * S]);
    {
      const HiLo<T> k1 = {p.cv4[T4_U1H], p.cv4[T4_U1L]}, k2 = {p.cv4[T4_U2H], p.cv4[T4_U2L]},
                    k3 = {p.cv4[T4_U3H], p.cv4[T4_U3L]}, ki = {p.cv4[T4_IUH], p.cv4[T4_IUL]};
      T rn[8];
      if (j - 7 >= ja) {
#pragma unroll
        for (int u = 0; u < 8; ++u) rn[u] = w_l[(size_t)(j - u) * S];
      }
      for (; j - 7 >= ja; j -= 8) {
        T r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = rn[u];
        if (j - 15 >= ja) {
#pragma unroll
          for (int u = 0; u < 8; ++u) rn[u] = w_l[(size_t)(j - 8 - u) * S];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) bstep(j - u, k1, k2, k3, ki, r[u]);
      }
      for (; j >= ja; --j) bstep(j, k1, k2, k3, ki, w_l[(size_t)j * S]);
    }
    for (; j >= 1; --j)
      bstep(j, tab(T4_U1H, j), tab(T4_U2H, j), tab(T4_U3H, j), tab(T4_IUH, j), w_l[(size_t)j * S]);
  }
  __syncthreads();
  // w at node m (-1 <= m <= N + 1) with odd images; zero on the walls
  auto wnode = [&](int m, int l) -> T {
    if (m <= 0 || m >= N) {
      if (m < 0 && -m < N) return -sW[(size_t)(-m) * S + l];
      if (m > N && 2 * N - m > 0) return -sW[(size_t)(2 * N - m) * S + l];
      return T(0);
    }
    return sW[(size_t)m * S + l];
  };
  // 4. H += kd D w at the faces, E <- alpha w + beta E at the nodes
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int j = 32 * c + jo;
    if (j >= N) continue;
    T hn[V], en[V];
    if constexpr (!ROWS) {
      // w at node m as a vector, with the odd images of wnode
      auto wrow = [&](int m, T* out) {
        T sg = T(1);
        int g = m;
        if (m <= 0 || m >= N) {
          sg = T(-1);
          g = (m < 0 && -m < N) ? -m : ((m > N && 2 * N - m > 0) ? 2 * N - m : -1);
        }
        if (g < 0) {
#pragma unroll
          for (int v = 0; v < V; ++v) out[v] = T(0);
        } else {
          ldrow(sW, g, out);
          if (sg < T(0)) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = -out[v];
          }
        }
      };
      T w0[V], wp[V], wp2[V], wm[V], h0[V];
      wrow(j, w0);
      wrow(j + 1, wp);
      wrow(j + 2, wp2);
      wrow(j - 1, wm);
      ldrow(sH, j, h0);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T dw = c1 * (wp[v] - w0[v]) + c2 * (wp2[v] - wm[v]);
        hn[v] = fma(p.kd, dw, h0[v]);
        en[v] = fma(p.alpha, w0[v], p.beta * Ev[c][v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int l = lv(v);
        const T dw = c1 * (wnode(j + 1, l) - wnode(j, l)) + c2 * (wnode(j + 2, l) - wnode(j - 1, l));
        hn[v] = fma(p.kd, dw, sH[(size_t)j * S + l]);
        const T w = (j >= 1) ? sW[(size_t)j * S + l] : T(0);
        en[v] = fma(p.alpha, w, p.beta * Ev[c][v]);
      }
    }
    if constexpr (!ROWS) {
      const long long at = s_base[lv(0)] + (long long)j * ls;
      if (all_ok) {
        if (FDTD_IN_RANGE(at, at + V, p.n_elem)) {
          *reinterpret_cast<VT*>(p.h_out + at) = vec16_make(hn);
          *reinterpret_cast<VT*>(p.e_out + at) = vec16_make(en);
        }
      } else if (any_ok) {
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (s_ok[lv(v)]) {
            p.h_out[at + v] = hn[v];
            p.e_out[at + v] = en[v];
          }
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int l = lv(v);
        if (s_ok[l]) {
          const long long at = s_base[l] + j;
          p.h_out[at] = hn[v];
          p.e_out[at] = en[v];
        }
      }
    }
  }
}

}  // namespace fdtd
