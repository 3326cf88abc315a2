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
// One thread per line walks it three times: the forward sweep of the banded
// LU (the right-hand side formed on the fly), the backward sweep, and the H
// and E updates; the intermediate values live in a field-shaped scratch
// array.  Lines along y and z take consecutive x on consecutive threads
// (coalesced); lines along x are rows.
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

}  // namespace fdtd
