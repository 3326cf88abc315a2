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
//   forward   y_j = r_j - m_j y_{j-1},           m_j = l_j / beta_{j-1}
//   backward  w_j = y_j / beta_j - c_j w_{j+1},  c_j = u_j / beta_j
// with 1/beta = 0 on wall nodes and beyond the line, which pins w = 0 there.
// Both recurrences are first-order linear, so a line is cut into segments:
// each thread runs the recurrences over its own segment from a zero carry,
// the segment carries are chained (a scan of affine maps x -> a + p x), and
// each thread adds carry * (product of its -m or -c) to its values.  This is
// the sequential Thomas result, reassociated; nothing is stored outside
// registers and a few words of shared memory.
//
// Coefficient sources (MODE): 0 = position tables of a homogeneous medium;
// 1 = the same tables' limit values, used on segments where the table is
// constant (the LU pivots of a constant-coefficient line converge
// geometrically, so past the first few nodes every entry equals its limit
// in working precision): kernel-parameter constants, no loads; 2 = per-node
// arrays of an inhomogeneous medium.
//
// Kernels:
//   proc_strided_kernel      lines along y or z, data loaded straight from HBM.
//   proc_strided_tma_kernel  the same lines, persistent: each block walks a
//                            list of tiles (LANES lines x all nodes) with the
//                            next tile's E and H streamed into shared memory
//                            by TMA (cp.async.bulk.tensor) while the current
//                            tile is solved, so HBM never waits on compute.
//   proc_rows_kernel         lines along x (contiguous): one warp per line,
//                            lane l owns nodes/faces [l L, l L + L) loaded as
//                            16-byte vectors; carries go through shuffles.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

// Bounds-checked debug build (-DFDTD_BOUNDS): every line, tile or element a
// kernel is about to touch is checked against its array's extent; a range
// outside it is recorded in g_bounds_err (read by the host's device-flag
// check, FDTD_ERR_BOUNDS) and the accesses are skipped.  Each check covers a
// whole line: its accesses are base + j ls for j in a known range, so the
// first and the last one bound the rest.  Without the macro the checks are
// the constant true.  TMA copies need none: the tensor map bounds them.
#ifdef FDTD_BOUNDS
__device__ int g_bounds_err = 0;
// [lo, hi) inside [0, n)?
__device__ __forceinline__ bool in_range(long long lo, long long hi, long long n) {
  if (lo >= 0 && lo <= hi && hi <= n) return true;
  atomicExch(&g_bounds_err, 1);
  return false;
}
#define FDTD_IN_RANGE(lo, hi, n) ::fdtd::in_range((lo), (hi), (n))
#else
#define FDTD_IN_RANGE(lo, hi, n) true
#endif

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
  int e_unit;            // alpha = 1, beta = -1 (the procedure's E <- w - E)
  const T* tab;          // uniform: [TB_ROWS][tlen] hi/lo rows of 1/beta, m, c and the
                         // segment carry products PF, PB (zero beyond N and at walls)
  int tlen;
  int jc;                // uniform: segments starting at j0 >= jc and ending by N are
                         // "converged": their coefficients are the constants below
  T cv[6];               // converged 1/beta, m, c as (hi, lo) pairs
  T qf[2][32];           // converged PF_t = (-m)^(t+1), hi and lo
  T qb[2][32];           // converged PB_t = (-c)^(L-t), hi and lo
  // per-node media, rows scaled by 1/b_j (symmetric form): r'_j = q_j E_j +
  // ks (H_j - H_{j-1}), constant off-diagonal off, pivots 1/beta_j (hi + lo)
  const T* nq;           // per-node: q_j = 1/|b_j| at each E node (field layout)
  const T* nib;          // per-node: 1/beta_j, hi part (field layout)
  const T* nibl;         // per-node: 1/beta_j, lo part (FP32 fields only)
  T ks;                  // per-node: RHS coupling of the scaled rows, s sign(h) / d_eta
  T offh, offl;          // per-node: off-diagonal -|ks| |kd| / 2 as hi + lo
  int* err;              // set to 1 when a bounded device wait gives up
  T* d_out;              // per-node kernels: when set, also E_in - E_out per E node
                         // (the reverse pass's record of the procedure)
  // per-node mu (general media): face f between nodes f and f+1 (stored at
  // node f) has its own H coupling kd_f = kd_scale * nkd[f] and off-diagonal
  // noffh[f] + noffl[f]; nullptr when mu is uniform
  const T* nkd;
  const T* noffh;
  const T* noffl;
  T kd_scale;
  long long n_elem;      // elements of every field-layout array (bounds-checked builds)
  int tables_only;       // uniform media: every lane reads the tables (no converged-
                         // constant branch); set for FP64 fields on large pairs
  int wall_fix;          // uniform media: solve with the converged factors on every
                         // lane plus the rank-one wall correction (table rows
                         // TB_KGH/TB_KGL) instead of table lanes near the walls
  int kg_len;            // the wall correction is zero from this node on (a multiple of
                         // the segment length)
  T* tmp4;               // fourth-order differences: field-shaped scratch of the line solve
  T c2_4;                // fourth-order difference weight -1/24 in the field precision
  int jc4, je4;          // fourth-order differences: the factor rows of nodes jc4..je4 all
                         // equal cv4 (empty when jc4 > je4)
  T cv4[14];             // those rows' (hi, lo) l1, l2, l3, 1/u0, u1, u2, u3
};

// Bounds of one line for the checked build: a strided line touches its
// nodes 0 .. N-1 at base + j ls; an x line (row) is read and written in
// whole segments of L elements from base, the last one holding node N-1.
template <typename T>
__device__ __forceinline__ bool strided_line_ok(const PairParams<T>& p, long long base) {
  return FDTD_IN_RANGE(base, base + (long long)(p.N - 1) * p.ls + 1, p.n_elem);
}
template <typename T, int L>
__device__ __forceinline__ bool row_ok(const PairParams<T>& p, long long base) {
  return FDTD_IN_RANGE(base, base + (long long)((p.N + L - 1) / L) * L, p.n_elem);
}

// ---------------------------------------------------------------------------
// Segment arithmetic shared by all kernels
// ---------------------------------------------------------------------------
// FP32 fields apply every FP64-formed coefficient as a pair hi + lo of FP32
// numbers (hi = the FP64 value rounded, lo = the rounded remainder): the
// solve then inverts the FP64-factored matrix to about 2^-48 instead of a
// matrix perturbed by the rounding of its pivots.  Rounded pivots perturb
// the diagonal of (1/2 I - h/4 O) identically at every step, which makes a
// procedure slightly non-unitary and the field energy drift steadily; with
// hi + lo the remaining error is the ordinary FP32 rounding of the fields.
// FP64 fields use the coefficients as they are (lo terms compile away).
template <typename T>
struct HiLo {
  T hi, lo;
};

template <typename T>
__device__ __forceinline__ constexpr bool use_hilo() {
  return sizeof(T) == 4;
}

// a * x + b with a = hi + lo
template <typename T>
__device__ __forceinline__ T fma2(HiLo<T> a, T x, T b) {
  if constexpr (use_hilo<T>()) return fma(a.hi, x, fma(a.lo, x, b));
  else return fma(a.hi, x, b);
}

// E_out = alpha w + beta E of a segment.  FP64 fields: the procedure's own
// E <- w - E (p.e_unit) is one subtraction; fma(1, w, -E) rounds w - E once,
// exactly as the subtraction does, so both forms give the same bits, with
// one FP64 instruction fewer per node where the FP64 pipe binds (the branch
// is the same for every thread of a launch).  FP32 fields keep the fused form:
// their kernels are bound by HBM, and the second path costs the x-line
// kernel 8 registers and 6 % of its time.
template <typename T, int L>
__device__ __forceinline__ void e_next(const PairParams<T>& p, const T (&y)[L], const T (&E)[L], T (&En)[L]) {
  if (sizeof(T) == 8 && p.e_unit) {
#pragma unroll
    for (int t = 0; t < L; ++t) En[t] = y[t] - E[t];
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) En[t] = fma(p.alpha, y[t], p.beta * E[t]);
  }
}

template <typename T, int L>
__device__ __forceinline__ void e_update(const PairParams<T>& p, const T (&y)[L], T (&E)[L]) {
  if (sizeof(T) == 8 && p.e_unit) {
#pragma unroll
    for (int t = 0; t < L; ++t) E[t] = y[t] - E[t];
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) E[t] = fma(p.alpha, y[t], p.beta * E[t]);
  }
}

// Table rows of a homogeneous medium, each [tlen] long.
// TB_KGH/TB_KGL: the rank-one wall correction kappa g_j of the constant-factor
// x-line solve (row_solve_store_wall), zero at node 0 and from node N on.
enum { TB_IBH = 0, TB_IBL, TB_MH, TB_ML, TB_CH, TB_CL, TB_PFH, TB_PFL, TB_PBH, TB_PBL, TB_KGH, TB_KGL, TB_ROWS };

template <typename T, int MODE>
__device__ __forceinline__ HiLo<T> tab2(const PairParams<T>& p, int row, int j, int t, const T* cv_hi,
                                        const T* cv_lo) {
  if constexpr (MODE == 0) return {p.tab[row * p.tlen + j], p.tab[(row + 1) * p.tlen + j]};
  else return {cv_hi[t], cv_lo[t]};
}

// a * b for a, b given as hi + lo (FP32 fields: error-free product of the
// hi parts plus the cross terms; FP64 fields: the plain product)
template <typename T>
__device__ __forceinline__ HiLo<T> dd_mul(HiLo<T> a, HiLo<T> b) {
  const T ph = a.hi * b.hi;
  if constexpr (use_hilo<T>()) {
    const T e = fma(a.hi, b.hi, -ph);
    return {ph, fma(a.hi, b.lo, fma(a.lo, b.hi, e))};
  } else {
    return {ph, T(0)};
  }
}

// Forward multiplier m, backward coupling c, pivot 1/beta of node j0 + t.
// Per-node media (MODE 2): ibn / ibl hold this segment's pivots (hi, lo),
// ib_prev the previous node's; m_j = off / beta_{j-1}, c_j = off / beta_j.
template <typename T, int L, int MODE>
__device__ __forceinline__ HiLo<T> coef_m(const PairParams<T>& p, int j0, int t, const T (&ibl)[L],
                                          const T (&ibn)[L], HiLo<T> ib_prev) {
  if constexpr (MODE == 0) return {p.tab[TB_MH * p.tlen + j0 + t], p.tab[TB_ML * p.tlen + j0 + t]};
  else if constexpr (MODE == 1) return {p.cv[2], p.cv[3]};
  else return dd_mul(HiLo<T>{p.offh, p.offl}, t == 0 ? ib_prev : HiLo<T>{ibn[t - 1], ibl[t - 1]});
}
template <typename T, int L, int MODE>
__device__ __forceinline__ HiLo<T> coef_c(const PairParams<T>& p, int j0, int t, const T (&ibl)[L],
                                          const T (&ibn)[L]) {
  if constexpr (MODE == 0) return {p.tab[TB_CH * p.tlen + j0 + t], p.tab[TB_CL * p.tlen + j0 + t]};
  else if constexpr (MODE == 1) return {p.cv[4], p.cv[5]};
  else return dd_mul(HiLo<T>{p.offh, p.offl}, HiLo<T>{ibn[t], ibl[t]});
}
template <typename T, int L, int MODE>
__device__ __forceinline__ HiLo<T> coef_ib(const PairParams<T>& p, int j0, int t, const T (&ibl)[L],
                                           const T (&ibn)[L]) {
  if constexpr (MODE == 0) return {p.tab[TB_IBH * p.tlen + j0 + t], p.tab[TB_IBL * p.tlen + j0 + t]};
  else if constexpr (MODE == 1) return {p.cv[0], p.cv[1]};
  else return {ibn[t], ibl[t]};
}
// Carry products within the segment: PF_t = prod_{u<=t} (-m_u), PB_t = prod_{u>=t} (-c_u).
template <typename T, int MODE>
__device__ __forceinline__ HiLo<T> coef_pf(const PairParams<T>& p, int j0, int t) {
  if constexpr (MODE == 0) return {p.tab[TB_PFH * p.tlen + j0 + t], p.tab[TB_PFL * p.tlen + j0 + t]};
  else return {p.qf[0][t], p.qf[1][t]};
}
template <typename T, int MODE>
__device__ __forceinline__ HiLo<T> coef_pb(const PairParams<T>& p, int j0, int t) {
  if constexpr (MODE == 0) return {p.tab[TB_PBH * p.tlen + j0 + t], p.tab[TB_PBL * p.tlen + j0 + t]};
  else return {p.qb[0][t], p.qb[1][t]};
}

// RHS and local forward sweep from a zero carry; returns the segment's carry
// coefficient prod(-m).
// qn: per-node q_j (MODE 2); ibn, ibl: per-node pivots (MODE 2).
template <typename T, int L, int MODE>
__device__ __forceinline__ HiLo<T> phase_forward(const PairParams<T>& p, int j0, const T (&E)[L], const T (&H)[L],
                                                 T hm1, const T (&qn)[L], const T (&ibn)[L], const T (&ibl)[L],
                                                 HiLo<T> ib_prev, T (&y)[L]) {
  T pf = T(1), hprev = hm1;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    T r;
    if constexpr (MODE == 2) r = fma(qn[t], E[t], p.ks * (H[t] - hprev));
    else r = fma(p.kb, H[t] - hprev, E[t]);
    hprev = H[t];
    if constexpr (MODE == 2 && use_hilo<T>()) {
      // FP32: m_t = off / beta_{t-1}: y_t = r_t - off (y_{t-1} / beta_{t-1}),
      // the pivot and the off-diagonal each applied as hi + lo (no
      // double-float product of the two).  FP64 keeps m_t = off * (1/beta)
      // as one product: fewer operations on the FP64 pipe that binds it.
      if (t == 0) {
        y[t] = r;
      } else {
        const T v = fma(ibn[t - 1], y[t - 1], ibl[t - 1] * y[t - 1]);
        y[t] = fma(-p.offh, v, fma(-p.offl, v, r));
      }
      pf *= -p.offh * (t == 0 ? ib_prev.hi : ibn[t - 1]);
    } else {
      const HiLo<T> m = coef_m<T, L, MODE>(p, j0, t, ibl, ibn, ib_prev);
      y[t] = (t == 0) ? r : fma2(HiLo<T>{-m.hi, -m.lo}, y[t - 1], r);
      if constexpr (MODE == 2) pf *= -m.hi;
    }
  }
  if constexpr (MODE == 2) return {pf, T(0)};
  else return coef_pf<T, MODE>(p, j0, L - 1);
}

// Forward carry fix-up, then the local backward sweep from a zero carry;
// returns the segment's carry coefficient prod(-c).
template <typename T, int L, int MODE>
__device__ __forceinline__ HiLo<T> phase_backward(const PairParams<T>& p, int j0, T yin, const T (&ibn)[L],
                                                  const T (&ibl)[L], HiLo<T> ib_prev, T (&y)[L]) {
  if constexpr (MODE == 2) {
    T q = T(1);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if constexpr (use_hilo<T>()) q *= -p.offh * (t == 0 ? ib_prev.hi : ibn[t - 1]);
      else q *= -coef_m<T, L, MODE>(p, j0, t, ibl, ibn, ib_prev).hi;
      y[t] = fma(q, yin, y[t]);
    }
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) y[t] = fma2(coef_pf<T, MODE>(p, j0, t), yin, y[t]);
  }
  T pb = T(1), wn = T(0);
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    if constexpr (MODE == 2 && use_hilo<T>()) {
      // FP32: c_t = off / beta_t: w_t = (y_t - off w_{t+1}) / beta_t
      const T u = fma(-p.offh, wn, fma(-p.offl, wn, y[t]));
      y[t] = fma(ibn[t], u, ibl[t] * u);
      pb *= -p.offh * ibn[t];
    } else {
      const HiLo<T> c = coef_c<T, L, MODE>(p, j0, t, ibl, ibn);
      const HiLo<T> ib = coef_ib<T, L, MODE>(p, j0, t, ibl, ibn);
      T u;
      if constexpr (use_hilo<T>()) u = fma(-c.hi, wn, fma(-c.lo, wn, y[t] * ib.lo));
      else u = -c.hi * wn;
      y[t] = fma(y[t], ib.hi, u);
      if constexpr (MODE == 2) pb *= -c.hi;
    }
    wn = y[t];
  }
  if constexpr (MODE == 2) return {pb, T(0)};
  else return coef_pb<T, MODE>(p, j0, 0);
}

// Backward carry fix-up: y becomes w.
template <typename T, int L, int MODE>
__device__ __forceinline__ void phase_fix(const PairParams<T>& p, int j0, T win, const T (&ibn)[L],
                                          const T (&ibl)[L], T (&y)[L]) {
  if constexpr (MODE == 2) {
    T q = T(1);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      if constexpr (use_hilo<T>()) q *= -p.offh * ibn[t];
      else q *= -coef_c<T, L, MODE>(p, j0, t, ibl, ibn).hi;
      y[t] = fma(q, win, y[t]);
    }
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) y[t] = fma2(coef_pb<T, MODE>(p, j0, t), win, y[t]);
  }
}

// Carry chains across the P segments of LANES lines.  Each chain is an
// inclusive scan over segments of the affine maps x -> a_q + p_q x, one scan
// per lane.  The (lane, segment) items are spread over groups of PW = 2^k >= P
// consecutive threads so the scan runs as a Kogge-Stone on warp shuffles with
// every thread of the block taking part (uniform trip count; the block size
// is a multiple of 32).  reverse = true scans from the last segment.  The
// first combine (a neighbour's carry) uses p as hi + lo; longer-range
// products are FP32 (their weight is already below prod(-m)^2 over a
// segment, far under the rounding of the result).
// tid, nthr: this thread's index among the nthr threads that own the lines
// (the whole block unless a block holds several tiles; nthr is a multiple
// of 32 and equal for every tile of the block, so trip counts match).
template <typename T, int LANES>
__device__ __forceinline__ void chain_scan(T* sa, const T* sph, const T* spl, int P, int PS, int PW, bool reverse,
                                           int tid, int nthr) {
  const unsigned FULL = 0xffffffffu;
  const int items = LANES * PW;
  for (int first = 0; first < items; first += nthr) {
    const int it = first + tid;
    const int lane = it / PW;
    const int q = it % PW;
    const bool valid = (it < items) && (q < P);
    const int qq = reverse ? (P - 1 - q) : q;
    const int at = lane * PS + qq;
    T a = valid ? sa[at] : T(0);
    T ph = valid ? sph[at] : T(1);
    const T pl = valid ? spl[at] : T(0);
    for (int d = 1; d < PW; d <<= 1) {
      const T au = __shfl_up_sync(FULL, a, d, PW);
      const T pu = __shfl_up_sync(FULL, ph, d, PW);
      if (q >= d) {
        a = (d == 1) ? fma2(HiLo<T>{ph, pl}, au, a) : fma(ph, au, a);
        ph = ph * pu;
      }
    }
    if (valid) sa[at] = a;
  }
}

// Chain buffers: [6][LANES][PS], PS = P rounded up to odd so that both the
// per-segment writes (lanes across a warp) and the scan reads (segments
// across a warp) are free of bank conflicts.
__device__ __forceinline__ int chain_stride(int P) { return P | 1; }

// Forward chain: returns y at the last node of segment s-1 (0 for s = 0).
template <typename T, int LANES>
__device__ __forceinline__ T block_chain_forward(T* sh, int P, int PW, int s, int lane, T a, HiLo<T> pm, int tid,
                                                 int nthr) {
  const int PS = chain_stride(P);
  T* sa = sh;
  T* sph = sh + PS * LANES;
  T* spl = sh + 2 * PS * LANES;
  sa[lane * PS + s] = a;
  sph[lane * PS + s] = pm.hi;
  spl[lane * PS + s] = pm.lo;
  __syncthreads();
  chain_scan<T, LANES>(sa, sph, spl, P, PS, PW, false, tid, nthr);
  __syncthreads();
  return (s > 0) ? sa[lane * PS + s - 1] : T(0);
}

// Backward chain: returns w at the first node of segment s+1 (0 for the last).
template <typename T, int LANES>
__device__ __forceinline__ T block_chain_backward(T* sh, int P, int PW, int s, int lane, T b, HiLo<T> pm, int tid,
                                                  int nthr) {
  const int PS = chain_stride(P);
  T* sa = sh + 3 * PS * LANES;
  T* sph = sh + 4 * PS * LANES;
  T* spl = sh + 5 * PS * LANES;
  sa[lane * PS + s] = b;
  sph[lane * PS + s] = pm.hi;
  spl[lane * PS + s] = pm.lo;
  __syncthreads();
  chain_scan<T, LANES>(sa, sph, spl, P, PS, PW, true, tid, nthr);
  __syncthreads();
  return (s + 1 < P) ? sa[lane * PS + s + 1] : T(0);
}

__device__ __forceinline__ int pow2_at_least(int P) {
  int w = 1;
  while (w < P) w <<= 1;
  return w;
}

// The whole segment solve of a block of LANES lines.  MODE may differ
// between warps; every barrier sits outside the MODE branches.
template <typename T, int LANES, int L, bool PER_NODE>
__device__ __forceinline__ void strided_solve(const PairParams<T>& p, int j0, int s, int P, int lane, T* sh,
                                              const T (&E)[L], const T (&H)[L], T hm1, const T (&qn)[L],
                                              const T (&ibn)[L], const T (&ibl)[L], HiLo<T> ib_prev, T (&y)[L],
                                              T& win, int tid = -1, int nthr = -1) {
  if (tid < 0) {
    tid = (int)threadIdx.x;
    nthr = (int)blockDim.x;
  }
  // p.tables_only (FP64 fields on large pairs): every lane reads the tables.
  // The converged constants equal the table entries, and a warp whose
  // segments took both branches would issue the FP64 arithmetic of both on
  // the FP64 pipe that bounds the solve
  const bool conv = !p.tables_only && (j0 >= p.jc) && (j0 + L <= p.N);
  HiLo<T> pf, pb;
  if constexpr (PER_NODE) {
    pf = phase_forward<T, L, 2>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
  } else {
    if (conv) pf = phase_forward<T, L, 1>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
    else pf = phase_forward<T, L, 0>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
  }
  const int PW = pow2_at_least(P);
  const T yin = block_chain_forward<T, LANES>(sh, P, PW, s, lane, y[L - 1], pf, tid, nthr);
  if constexpr (PER_NODE) {
    pb = phase_backward<T, L, 2>(p, j0, yin, ibn, ibl, ib_prev, y);
  } else {
    if (conv) pb = phase_backward<T, L, 1>(p, j0, yin, ibn, ibl, ib_prev, y);
    else pb = phase_backward<T, L, 0>(p, j0, yin, ibn, ibl, ib_prev, y);
  }
  win = block_chain_backward<T, LANES>(sh, P, PW, s, lane, y[0], pb, tid, nthr);
  if constexpr (PER_NODE) {
    phase_fix<T, L, 2>(p, j0, win, ibn, ibl, y);
  } else {
    if (conv) phase_fix<T, L, 1>(p, j0, win, ibn, ibl, y);
    else phase_fix<T, L, 0>(p, j0, win, ibn, ibl, y);
  }
}

// The segment solve of a block of LANES lines of a homogeneous medium with
// the converged factors on every segment and the rank-one wall correction
// (the strided counterpart of row_solve_store_wall): no segment reads the
// factor tables, so every warp runs the same arithmetic between the chain
// barriers.  Node 1's value w'_1 of every line reaches the segments that need
// it without another barrier: segment 0 publishes its local backward value
// there in a slot of the forward chain buffers that is free by then, and
// every thread adds segment 0's incoming backward carry after the chain.  win
// comes back corrected too (the next segment's first node).
template <typename T, int LANES, int L>
__device__ __forceinline__ void strided_solve_wall(const PairParams<T>& p, int j0, int s, int P, int lane, T* sh,
                                                   const T (&E)[L], const T (&H)[L], T hm1, T (&y)[L], T& win,
                                                   int tid = -1, int nthr = -1) {
  if (tid < 0) {
    tid = (int)threadIdx.x;
    nthr = (int)blockDim.x;
  }
  const int N = p.N;
  const HiLo<T> m = {p.cv[2], p.cv[3]};
  const HiLo<T> ib = {p.cv[0], p.cv[1]};
  const HiLo<T> c = {p.cv[4], p.cv[5]};
  T hprev = hm1;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    T r = fma(p.kb, H[t] - hprev, E[t]);
    hprev = H[t];
    if (t == 0) r = (j0 == 0) ? T(0) : r;  // node 0 (past the end: cut off below)
    y[t] = (t == 0) ? r : fma2(HiLo<T>{-m.hi, -m.lo}, y[t - 1], r);
  }
  const int PW = pow2_at_least(P);
  const T yin = block_chain_forward<T, LANES>(sh, P, PW, s, lane, y[L - 1], HiLo<T>{p.qf[0][L - 1], p.qf[1][L - 1]},
                                              tid, nthr);
#pragma unroll
  for (int t = 0; t < L; ++t) y[t] = fma2(HiLo<T>{p.qf[0][t], p.qf[1][t]}, yin, y[t]);
  const bool full = j0 + L <= N;
  T wn = T(0);
  if (full) {
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      T u;
      if constexpr (use_hilo<T>()) u = fma(-c.hi, wn, fma(-c.lo, wn, y[t] * ib.lo));
      else u = -c.hi * wn;
      y[t] = fma(y[t], ib.hi, u);
      wn = y[t];
    }
  } else {
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      const bool in = j0 + t < N;
      const T ch = in ? c.hi : T(0), cl = in ? c.lo : T(0);
      const T ih = in ? ib.hi : T(0), il = in ? ib.lo : T(0);
      T u;
      if constexpr (use_hilo<T>()) u = fma(-ch, wn, fma(-cl, wn, y[t] * il));
      else u = -ch * wn;
      y[t] = fma(y[t], ih, u);
      wn = y[t];
    }
  }
  // segment 0 publishes node 1's local value in the forward chain's slot of
  // segment 0's hi products (read there only inside the forward scan)
  const int PS = chain_stride(P);
  T* ys1 = sh + PS * LANES;  // [lane * PS]
  if (s == 0) ys1[lane * PS] = (L >= 2) ? y[1 % L] : T(0);
  const HiLo<T> pb0 = full ? HiLo<T>{p.qb[0][0], p.qb[1][0]} : HiLo<T>{T(0), T(0)};
  win = block_chain_backward<T, LANES>(sh, P, PW, s, lane, y[0], pb0, tid, nthr);
  if (full) {
#pragma unroll
    for (int t = 0; t < L; ++t) y[t] = fma2(HiLo<T>{p.qb[0][t], p.qb[1][t]}, win, y[t]);
  }
  if (j0 == 0) y[0] = T(0);  // node 0: the wall
  if (j0 < p.kg_len) {
    // w'_1 = segment 0's local value + its carry-product times its incoming
    // backward carry (the chain result at segment 1)
    const T* sab = sh + 3 * PS * LANES;
    const T win0 = (P > 1) ? sab[lane * PS + 1] : T(0);
    const bool full0 = L <= N;
    const HiLo<T> pb1 = full0 ? HiLo<T>{p.qb[0][1 % L], p.qb[1][1 % L]} : HiLo<T>{T(0), T(0)};
    const T w1 = fma2(pb1, win0, ys1[lane * PS]);
    const T* kgh = p.tab + TB_KGH * p.tlen + j0;
    const T* kgl = p.tab + TB_KGL * p.tlen + j0;
#pragma unroll
    for (int t = 0; t < L; ++t) y[t] = fma2(HiLo<T>{kgh[t], kgl[t]}, w1, y[t]);
    win = fma2(HiLo<T>{kgh[L], kgl[L]}, w1, win);
  }
}

// Lines along y or z of a homogeneous medium, FP64 fields: one thread per
// line walks the strided axis (consecutive x on consecutive threads, every
// access coalesced) through the plain Thomas recurrences with the tabulated
// factors, the forward values in a field-shaped scratch array ys:
//   y_j = r_j - m_j y_{j-1},   w_j = (1/beta_j) y_j - c_j w_{j+1},
// then H_j += kd (w_{j+1} - w_j) and E_j <- alpha w_j + beta E_j as w_j
// appears.  Per node 8 FP64 instructions against the segmented solve's 10
// and its carry scans: the FP64 pipe binds these lines, and a launch of
// 256 x 255 lines still keeps it busy.  Reads of E and H happen before any
// write of the same line (in place is safe).  Chunks of SEQ_U = 8 nodes
// (97 registers) measured faster than 16 (196 registers: 8.1 against 8.5 G
// cell-steps/s at 256^3).  x lines keep the segmented solve: a thread per
// row, its lanes a row pitch apart, measured slower (6.6 against 8.4 G).
template <typename T, bool PER_NODE, int SEQ_U = 8>
__global__ void __launch_bounds__(128) proc_strided_seq_kernel(const PairParams<T> p, T* __restrict__ ys) {
  const long long nl = p.lane_hi - p.lane_lo;
  const long long line = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (nl <= 0 || line >= nl * p.n_o) return;
  const int i = p.lane_lo + (int)(line % nl);
  const int o = p.o_lo + (int)(line / nl);
  const long long base = (long long)o * p.os + i;
  if (!strided_line_ok(p, base)) return;
  const int N = p.N;
  const long long ls = p.ls;
  // homogeneous media: tabulated m_j, 1/beta_j, c_j; per-node media (rows
  // scaled by 1/b_j): r_j = q_j E_j + ks (H_j - H_{j-1}), m_j = off / beta_{j-1},
  // c_j = off / beta_j from the per-node pivots, as in the segmented solve
  const T* tm = p.tab + TB_MH * p.tlen;
  const T* tib = p.tab + TB_IBH * p.tlen;
  const T* tc = p.tab + TB_CH * p.tlen;
  // forward sweep over the unknowns 1 .. N-1 (nodes 0 and N are the walls),
  // in chunks of U nodes whose loads are all issued before their arithmetic
  // (the stores to ys may alias the field arrays as far as the compiler
  // knows, so it would not move later loads above them)
  constexpr int U = SEQ_U;
  T hprev = p.h_in[base];
  T yprev = T(0);
  T ibprev = PER_NODE ? p.nib[base] : T(0);
  for (int j0 = 1; j0 < N; j0 += U) {
    T hv[U], ev[U], mv[U], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j < N) {
        const long long at = base + (long long)j * ls;
        hv[u] = p.h_in[at];
        ev[u] = p.e_in[at];
        if constexpr (PER_NODE) {
          qv[u] = p.nq[at];
          mv[u] = p.nib[at];  // 1/beta_j: m_{j+1} = off / beta_j
        } else {
          mv[u] = __ldg(tm + j);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u;
      if (j < N) {
        T r, m;
        if constexpr (PER_NODE) {
          r = fma(qv[u], ev[u], p.ks * (hv[u] - hprev));
          m = p.offh * ibprev;
          ibprev = mv[u];
        } else {
          r = fma(p.kb, hv[u] - hprev, ev[u]);
          m = mv[u];
        }
        hprev = hv[u];
        const T y = fma(-m, yprev, r);
        ys[base + (long long)j * ls] = y;
        yprev = y;
      }
    }
  }
  // backward sweep with the H and E updates of each node as its w appears
  const bool unit = p.e_unit != 0;
  T wnext = T(0);
  for (int j1 = N - 1; j1 >= 1; j1 -= U) {
    T yv[U], hv[U], ev[U], bv[U], cv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j1 - u;
      if (j >= 1) {
        const long long at = base + (long long)j * ls;
        yv[u] = ys[at];
        hv[u] = p.h_in[at];
        ev[u] = p.e_in[at];
        if constexpr (PER_NODE) {
          bv[u] = p.nib[at];
        } else {
          bv[u] = __ldg(tib + j);
          cv[u] = __ldg(tc + j);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j1 - u;
      if (j >= 1) {
        const long long at = base + (long long)j * ls;
        const T c = PER_NODE ? p.offh * bv[u] : cv[u];
        const T w = fma(yv[u], bv[u], -c * wnext);
        p.h_out[at] = fma(p.kd, wnext - w, hv[u]);
        p.e_out[at] = unit ? w - ev[u] : fma(p.alpha, w, p.beta * ev[u]);
        wnext = w;
      }
    }
  }
  // face 0 (w_0 = 0) and the wall node 0
  p.h_out[base] = fma(p.kd, wnext - T(0), p.h_in[base]);
  const T e0 = p.e_in[base];
  p.e_out[base] = unit ? T(0) - e0 : fma(p.alpha, T(0), p.beta * e0);
}

// H update, subtraction and store of one strided segment.
template <typename T, int L>
__device__ __forceinline__ void strided_store(const PairParams<T>& p, long long base, int j0, const T (&E)[L],
                                              const T (&H)[L], const T (&y)[L], T win) {
  T* pe = p.e_out + base + (long long)j0 * p.ls;
  T* ph = p.h_out + base + (long long)j0 * p.ls;
  const long long ls = p.ls;
  T En[L];
  e_next<T, L>(p, y, E, En);
  if (j0 + L <= p.N) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T wnext = (t + 1 < L) ? y[t + 1] : win;
      pe[t * ls] = En[t];
      ph[t * ls] = fma(p.kd, wnext - y[t], H[t]);
    }
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t < p.N) {
        const T wnext = (t + 1 < L) ? y[t + 1] : win;
        pe[t * ls] = En[t];
        ph[t * ls] = fma(p.kd, wnext - y[t], H[t]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Lines along y or z, loads straight from HBM
// ---------------------------------------------------------------------------
template <typename T, int LANES, int L, bool PER_NODE>
__global__ void proc_strided_kernel(const PairParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sh = reinterpret_cast<T*>(smem_raw);  // [6][LANES][P|1]
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

  T E[L], H[L], y[L], qn[L], ibn[L], ibl[L];
  HiLo<T> ib_prev = {T(0), T(0)};
  T hm1 = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    qn[t] = T(0);
    ibn[t] = T(0);
    ibl[t] = T(0);
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
        if constexpr (PER_NODE) {
          qn[t] = p.nq[base + (long long)j * ls];
          ibn[t] = p.nib[base + (long long)j * ls];
          if constexpr (use_hilo<T>()) ibl[t] = p.nibl[base + (long long)j * ls];
        }
      }
    }
    if (j0 > 0 && j0 - 1 < N) {
      hm1 = ph[(long long)(j0 - 1) * ls];
      if constexpr (PER_NODE) {
        ib_prev.hi = p.nib[base + (long long)(j0 - 1) * ls];
        if constexpr (use_hilo<T>()) ib_prev.lo = p.nibl[base + (long long)(j0 - 1) * ls];
      }
    }
  }
  T win;
  if constexpr (!PER_NODE) {
    if (p.wall_fix) strided_solve_wall<T, LANES, L>(p, j0, s, P, lane, sh, E, H, hm1, y, win);
    else strided_solve<T, LANES, L, false>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, ib_prev, y, win);
  } else {
    strided_solve<T, LANES, L, true>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, ib_prev, y, win);
  }
  if (active) strided_store<T, L>(p, base, j0, E, H, y, win);
  if constexpr (PER_NODE) {
    if (active && p.d_out) {
#pragma unroll
      for (int t = 0; t < L; ++t)
        if (j0 + t < N) p.d_out[base + (long long)(j0 + t) * ls] = E[t] - fma(p.alpha, y[t], p.beta * E[t]);
    }
  }
}

// ---------------------------------------------------------------------------
// Lines along y or z, persistent, TMA-fed (homogeneous media)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for an mbarrier phase for at most limit_ns; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// Self-test of the bounded waits: an mbarrier that expects one arrival;
// with arrive = 0 nobody arrives, the wait gives up after limit_ns and the
// kernel reports it through *flag (1), as the TMA kernels do through their
// error flag; with arrive = 1 thread 0 arrives first and the wait succeeds.
__global__ void bounded_wait_probe_kernel(int* flag, unsigned long long limit_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive_expect_tx(&bar, 0);
    *flag = mbar_wait_bounded(&bar, 0, limit_ns) ? 0 : 1;
  }
}

struct TmaTiles {
  int BN;        // nodes per box (>= N, a multiple of 8, <= 256)
  int zbox;      // 0: box {LANES, BN, 1} (lines along y); 1: box {LANES, 1, BN} (along z)
  int tiles_x;   // ceil(lane_hi / LANES)
  int n_tiles;   // tiles_x * n_o
};

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// Dynamic shared memory: [NST stages][E, H][BN][LANES] + [6][LANES][P|1] + NST mbarriers.
// At most 256 nodes per line, so at most ceil(256 / L) segments of LANES threads;
// MINB blocks share an SM so that one block's barriers overlap another's work.
// Tile k of a block uses stage k % NST; its copy is issued NST tiles ahead.
template <typename T, int LANES, int L, int MINB, int NST>
__global__ void __launch_bounds__(LANES * ((256 + L - 1) / L), MINB)
    proc_strided_tma_kernel(const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmH,
                            const PairParams<T> p, const TmaTiles q) {
  static_assert(NST >= 2 && NST <= 4, "ring depth");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x % LANES;
  const int s = threadIdx.x / LANES;
  const int P = blockDim.x / LANES;
  const int stage_elems = q.BN * LANES;
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* sh = buf + 2 * NST * stage_elems;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sh + 6 * chain_stride(P) * LANES);
  const uint32_t stage_bytes = 2u * (uint32_t)stage_elems * (uint32_t)sizeof(T);
  const int j0 = s * L;
  const int N = p.N;

  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st) mbar_init(&bars[st], 1);
    mbar_fence_init();
  }
  __syncthreads();

  auto issue = [&](int tile, int stage) {
    const int x0 = (tile % q.tiles_x) * LANES;
    const int o = p.o_lo + tile / q.tiles_x;
    T* dE = buf + (2 * stage + 0) * stage_elems;
    T* dH = buf + (2 * stage + 1) * stage_elems;
    mbar_arrive_expect_tx(&bars[stage], stage_bytes);
    if (q.zbox) {
      tma_load_3d(dE, &tmE, &bars[stage], x0, o, 0);
      tma_load_3d(dH, &tmH, &bars[stage], x0, o, 0);
    } else {
      tma_load_3d(dE, &tmE, &bars[stage], x0, 0, o);
      tma_load_3d(dH, &tmH, &bars[stage], x0, 0, o);
    }
  };
  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st)
      if ((int)blockIdx.x + st * (int)gridDim.x < q.n_tiles) issue(blockIdx.x + st * gridDim.x, st);
  }

  uint32_t parity = 0;  // bit st: phase parity expected next on stage st
  int k = 0;
  for (int tile = blockIdx.x; tile < q.n_tiles; tile += gridDim.x, ++k) {
    const int stage = k % NST;
    if (!mbar_wait_bounded(&bars[stage], (parity >> stage) & 1u, kWaitLimitNs)) {
      // Give up: flag it, then drain before the block's shared memory is
      // released.  The timed-out stage's own bulk copy may still be in
      // flight, so it gets a second bounded wait; then the other stages'
      // copies (if any) land.  A copy still outstanding after that second
      // limit is left in flight; the host reports FDTD_ERR_TIMEOUT and the
      // step's results are not valid.
      if (threadIdx.x == 0) atomicExch(p.err, 1);
      mbar_wait_bounded(&bars[stage], (parity >> stage) & 1u, kWaitLimitNs);
      for (int d = 1; d < NST; ++d) {
        const int other = tile + d * (int)gridDim.x;
        const int st = (k + d) % NST;
        if (other < q.n_tiles) mbar_wait_bounded(&bars[st], (parity >> st) & 1u, kWaitLimitNs);
      }
      return;
    }
    parity ^= 1u << stage;

    const int x0 = (tile % q.tiles_x) * LANES;
    const int o = p.o_lo + tile / q.tiles_x;
    const int i = x0 + lane;
    const long long base = (long long)o * p.os + i;
    const bool active = (i >= p.lane_lo) && (i < p.lane_hi) && strided_line_ok(p, base);

    const T* sE = buf + (2 * stage + 0) * stage_elems;
    const T* sH = buf + (2 * stage + 1) * stage_elems;
    T E[L], H[L], y[L], qn[L], ibn[L], ibl[L];
#pragma unroll
    for (int t = 0; t < L; ++t) {
      qn[t] = T(0);
      ibn[t] = T(0);
      ibl[t] = T(0);
    }
    if (j0 + L <= N) {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        E[t] = sE[(j0 + t) * LANES + lane];
        H[t] = sH[(j0 + t) * LANES + lane];
      }
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const int j = j0 + t;
        const bool in = j < N;
        E[t] = in ? sE[j * LANES + lane] : T(0);
        H[t] = in ? sH[j * LANES + lane] : T(0);
      }
    }
    const T hm1 = (j0 > 0 && j0 - 1 < N) ? sH[(j0 - 1) * LANES + lane] : T(0);
    __syncthreads();  // this stage's buffer is free again
    if (threadIdx.x == 0) {
      const int next = tile + NST * (int)gridDim.x;
      if (next < q.n_tiles) {
        fence_proxy_async_smem();
        issue(next, stage);
      }
    }
    T win;
    if (p.wall_fix)
      strided_solve_wall<T, LANES, L>(p, j0, s, P, lane, sh, E, H, hm1, y, win);
    else
      strided_solve<T, LANES, L, false>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, HiLo<T>{T(0), T(0)}, y,
                                      win);
    if (active) strided_store<T, L>(p, base, j0, E, H, y, win);
  }
}

// TMA tensor store of one box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the committed stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the committed stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// The TMA-fed y/z kernel with its outputs staged in shared memory and written
// by TMA tensor stores of the same boxes, overlapped with the next tile.
// Shared memory: [NST stages][E, H][BN][LANES] + [E, H][BN][LANES] output +
// [6][LANES][P|1] + NST mbarriers.  The output box is written whole: lanes
// outside [lane_lo, lane_hi) write back the values they loaded, and nodes
// at or past the line end write zeros (the far-wall E and the unused H row
// beyond the last face are zero); parts of the box outside the array are
// clipped by the TMA unit.
template <typename T, int LANES, int L, int MINB, int NST>
__global__ void __launch_bounds__(LANES * ((256 + L - 1) / L), MINB)
    proc_strided_tma_st_kernel(const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmH,
                               const PairParams<T> p, const TmaTiles q) {
  static_assert(NST >= 2 && NST <= 4, "ring depth");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x % LANES;
  const int s = threadIdx.x / LANES;
  const int P = blockDim.x / LANES;
  const int stage_elems = q.BN * LANES;
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* oE = buf + 2 * NST * stage_elems;
  T* oH = oE + stage_elems;
  T* sh = oH + stage_elems;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sh + 6 * chain_stride(P) * LANES);
  const uint32_t stage_bytes = 2u * (uint32_t)stage_elems * (uint32_t)sizeof(T);
  const int j0 = s * L;
  const int N = p.N;

  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st) mbar_init(&bars[st], 1);
    mbar_fence_init();
  }
  __syncthreads();

  auto coords = [&](int tile, int& x0, int& o) {
    x0 = (tile % q.tiles_x) * LANES;
    o = p.o_lo + tile / q.tiles_x;
  };
  auto issue = [&](int tile, int stage) {
    int x0, o;
    coords(tile, x0, o);
    T* dE = buf + (2 * stage + 0) * stage_elems;
    T* dH = buf + (2 * stage + 1) * stage_elems;
    mbar_arrive_expect_tx(&bars[stage], stage_bytes);
    if (q.zbox) {
      tma_load_3d(dE, &tmE, &bars[stage], x0, o, 0);
      tma_load_3d(dH, &tmH, &bars[stage], x0, o, 0);
    } else {
      tma_load_3d(dE, &tmE, &bars[stage], x0, 0, o);
      tma_load_3d(dH, &tmH, &bars[stage], x0, 0, o);
    }
  };
  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st)
      if ((int)blockIdx.x + st * (int)gridDim.x < q.n_tiles) issue(blockIdx.x + st * gridDim.x, st);
  }

  uint32_t parity = 0;  // bit st: phase parity expected next on stage st
  int k = 0;
  for (int tile = blockIdx.x; tile < q.n_tiles; tile += gridDim.x, ++k) {
    const int stage = k % NST;
    if (!mbar_wait_bounded(&bars[stage], (parity >> stage) & 1u, kWaitLimitNs)) {
      // Give up: flag it, drain as the register-store kernel does (a second
      // bounded wait on the timed-out stage, then the other stages' copies),
      // let our own stores land, return.
      if (threadIdx.x == 0) atomicExch(p.err, 1);
      mbar_wait_bounded(&bars[stage], (parity >> stage) & 1u, kWaitLimitNs);
      for (int d = 1; d < NST; ++d) {
        const int other = tile + d * (int)gridDim.x;
        const int st = (k + d) % NST;
        if (other < q.n_tiles) mbar_wait_bounded(&bars[st], (parity >> st) & 1u, kWaitLimitNs);
      }
      if (threadIdx.x == 0) bulk_wait_all();
      return;
    }
    parity ^= 1u << stage;

    int x0, o;
    coords(tile, x0, o);
    const int i = x0 + lane;
    const bool active = (i >= p.lane_lo) && (i < p.lane_hi);

    const T* sE = buf + (2 * stage + 0) * stage_elems;
    const T* sH = buf + (2 * stage + 1) * stage_elems;
    T E[L], H[L], y[L], qn[L], ibn[L], ibl[L];
#pragma unroll
    for (int t = 0; t < L; ++t) {
      qn[t] = T(0);
      ibn[t] = T(0);
      ibl[t] = T(0);
    }
    if (j0 + L <= N) {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        E[t] = sE[(j0 + t) * LANES + lane];
        H[t] = sH[(j0 + t) * LANES + lane];
      }
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const int j = j0 + t;
        const bool in = j < N;
        E[t] = in ? sE[j * LANES + lane] : T(0);
        H[t] = in ? sH[j * LANES + lane] : T(0);
      }
    }
    const T hm1 = (j0 > 0 && j0 - 1 < N) ? sH[(j0 - 1) * LANES + lane] : T(0);
    if (threadIdx.x == 0) bulk_wait_read_all();  // the previous tile's stores have read the output buffer
    __syncthreads();  // this stage's buffer and the output buffer are free
    if (threadIdx.x == 0) {
      const int next = tile + NST * (int)gridDim.x;
      if (next < q.n_tiles) {
        fence_proxy_async_smem();
        issue(next, stage);
      }
    }
    T win;
    if (p.wall_fix)
      strided_solve_wall<T, LANES, L>(p, j0, s, P, lane, sh, E, H, hm1, y, win);
    else
      strided_solve<T, LANES, L, false>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, HiLo<T>{T(0), T(0)}, y,
                                      win);
    T En[L];
    e_next<T, L>(p, y, E, En);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < q.BN) {
        T eo = E[t], ho = H[t];
        if (active && j < N) {
          const T wnext = (t + 1 < L) ? y[t + 1] : win;
          eo = En[t];
          ho = fma(p.kd, wnext - y[t], H[t]);
        }
        oE[j * LANES + lane] = eo;
        oH[j * LANES + lane] = ho;
      }
    }
    fence_proxy_async_smem();  // the output writes, seen by the TMA unit
    __syncthreads();
    if (threadIdx.x == 0) {
      if (q.zbox) {
        tma_store_3d(&tmE, oE, x0, o, 0);
        tma_store_3d(&tmH, oH, x0, o, 0);
      } else {
        tma_store_3d(&tmE, oE, x0, 0, o);
        tma_store_3d(&tmH, oH, x0, 0, o);
      }
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
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

// Segment carry chain across the 32 lanes of a warp (x lines): inclusive
// scan of x -> a + p x; the first combine uses the neighbour's p as hi + lo.
template <typename T>
__device__ __forceinline__ T warp_chain_forward(T a, HiLo<T> pm) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  T pp = pm.hi;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T a_up = __shfl_up_sync(FULL, a, d);
    const T p_up = __shfl_up_sync(FULL, pp, d);
    if (lane >= d) {
      a = (d == 1) ? fma2(HiLo<T>{pp, pm.lo}, a_up, a) : fma(pp, a_up, a);
      pp = pp * p_up;
    }
  }
  T yin = __shfl_up_sync(FULL, a, 1);
  return lane == 0 ? T(0) : yin;
}

template <typename T>
__device__ __forceinline__ T warp_chain_backward(T b, HiLo<T> pm) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  T qq = pm.hi;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T b_dn = __shfl_down_sync(FULL, b, d);
    const T q_dn = __shfl_down_sync(FULL, qq, d);
    if (lane + d < 32) {
      b = (d == 1) ? fma2(HiLo<T>{qq, pm.lo}, b_dn, b) : fma(qq, b_dn, b);
      qq = qq * q_dn;
    }
  }
  T win = __shfl_down_sync(FULL, b, 1);
  return lane == 31 ? T(0) : win;
}

// One x line (a warp): solve and store.  E, H (and per-node qn, ibn, ibl)
// hold the line's segment of this lane, zero past the line end.
template <typename T, int L, bool PER_NODE>
__device__ __forceinline__ void row_solve_store(const PairParams<T>& p, long long line, T (&E)[L], T (&H)[L],
                                                const T (&qn)[L], const T (&ibn)[L], const T (&ibl)[L]) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const bool ok = row_ok<T, L>(p, base);
  const int j0 = lane * L;
  const int N = p.N;
  T y[L];

  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1);
  if (lane == 0) hm1 = T(0);
  HiLo<T> ib_prev = {T(0), T(0)};
  if constexpr (PER_NODE) {
    ib_prev.hi = __shfl_up_sync(FULL, ibn[L - 1], 1);
    if constexpr (use_hilo<T>()) ib_prev.lo = __shfl_up_sync(FULL, ibl[L - 1], 1);
    if (lane == 0) ib_prev = {T(0), T(0)};
  }

  if constexpr (PER_NODE) {
    const HiLo<T> pf = phase_forward<T, L, 2>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
    const T yin = warp_chain_forward<T>(y[L - 1], pf);
    const HiLo<T> pb = phase_backward<T, L, 2>(p, j0, yin, ibn, ibl, ib_prev, y);
    const T win = warp_chain_backward<T>(y[0], pb);
    phase_fix<T, L, 2>(p, j0, win, ibn, ibl, y);
    // H update and subtraction below use y (= w) and win
    T D[L], En[L];
    e_next<T, L>(p, y, E, En);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T wnext = (t + 1 < L) ? y[t + 1] : win;
      H[t] = fma(p.kd, wnext - y[t], H[t]);
      D[t] = E[t] - En[t];
      E[t] = En[t];
    }
    if (p.d_out && ok) {
      if (j0 + L <= N) {
        store_seg<T, L>(p.d_out + base + j0, D);
      } else {
#pragma unroll
        for (int t = 0; t < L; ++t)
          if (j0 + t < N) p.d_out[base + j0 + t] = D[t];
      }
    }
  } else {
    // homogeneous media: lanes in the converged interior use the limit
    // constants, lanes near the walls read the tables (with p.tables_only
    // every lane reads the tables, as in strided_solve)
    const bool conv = !p.tables_only && (j0 >= p.jc) && (j0 + L <= N);
    HiLo<T> pf, pb;
    if (conv) pf = phase_forward<T, L, 1>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
    else pf = phase_forward<T, L, 0>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
    const T yin = warp_chain_forward<T>(y[L - 1], pf);
    if (conv) pb = phase_backward<T, L, 1>(p, j0, yin, ibn, ibl, ib_prev, y);
    else pb = phase_backward<T, L, 0>(p, j0, yin, ibn, ibl, ib_prev, y);
    const T win = warp_chain_backward<T>(y[0], pb);
    if (conv) phase_fix<T, L, 1>(p, j0, win, ibn, ibl, y);
    else phase_fix<T, L, 0>(p, j0, win, ibn, ibl, y);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const T wnext = (t + 1 < L) ? y[t + 1] : win;
      H[t] = fma(p.kd, wnext - y[t], H[t]);
    }
    e_update<T, L>(p, y, E);
  }
  // values beyond N are exactly zero, so whole segments inside the padded
  // row are stored as vectors; the segment holding the line end element-wise
  if (!ok) return;
  if (j0 + L <= N) {
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
  } else if (j0 < N) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t < N) {
        p.e_out[base + j0 + t] = E[t];
        p.h_out[base + j0 + t] = H[t];
      }
    }
  }
}

// One x line of a homogeneous medium without divergent lanes.  The line
// matrix T (nodes 1..N-1) has LU factors that vary only near node 1 and
// converge to constants; the constant factors L' U' are the exact LU of
// T' = T + delta e_1 e_1^T (delta = beta_inf - T_11, a change of the first
// diagonal entry only).  So every lane solves T' w' = r with the converged
// constants (kernel parameters, no table loads), and the Sherman-Morrison
// formula restores T^{-1} r = w' + kappa g w'_1 with g = T'^{-1} e_1 and
// kappa = delta / (1 - delta g_1): one broadcast of w'_1 and one hi + lo FMA
// per node with kappa g_j from the table (it decays geometrically from the
// wall; zero at node 0 and from node N on).  Node 0 and nodes >= N carry no
// unknown: their right-hand side is zero, their factors 1/beta and c zero,
// and node 0 is set to zero after the solve.  The result equals the
// table-factor solve up to rounding (not bit for bit).
template <typename T, int L, bool FULL_LINE = false>
__device__ __forceinline__ void row_solve_store_wall(const PairParams<T>& p, long long line, T (&E)[L],
                                                     T (&H)[L]) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const bool ok = row_ok<T, L>(p, base);
  const int j0 = lane * L;
  const int N = p.N;
  // the wall correction of this lane's nodes (vector loads; cache-resident)
  T kgh[L], kgl[L];
  load_seg<T, L>(p.tab + TB_KGH * p.tlen + j0, kgh);
  load_seg<T, L>(p.tab + TB_KGL * p.tlen + j0, kgl);
  T y[L];
  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1);
  if (lane == 0) hm1 = T(0);
  const HiLo<T> m = {p.cv[2], p.cv[3]};
  const HiLo<T> ib = {p.cv[0], p.cv[1]};
  const HiLo<T> c = {p.cv[4], p.cv[5]};
  // forward sweep with the constant multiplier
  T hprev = hm1;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const int j = j0 + t;
    T r = fma(p.kb, H[t] - hprev, E[t]);
    hprev = H[t];
    if constexpr (FULL_LINE) {
      if (t == 0) r = (lane == 0) ? T(0) : r;  // node 0: the wall
    } else {
      r = (j == 0 || j >= N) ? T(0) : r;
    }
    y[t] = (t == 0) ? r : fma2(HiLo<T>{-m.hi, -m.lo}, y[t - 1], r);
  }
  const T yin = warp_chain_forward<T>(y[L - 1], HiLo<T>{p.qf[0][L - 1], p.qf[1][L - 1]});
#pragma unroll
  for (int t = 0; t < L; ++t) y[t] = fma2(HiLo<T>{p.qf[0][t], p.qf[1][t]}, yin, y[t]);
  // backward sweep; nodes >= N hold w = 0 and do not couple (masks by
  // selects: one code path keeps the kernel at 48 registers, where two
  // paths needed 64 and ran slower)
  const bool full = FULL_LINE || j0 + L <= N;
  T wn = T(0);
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    const bool in = FULL_LINE || j0 + t < N;
    const T ch = in ? c.hi : T(0), cl = in ? c.lo : T(0);
    const T ih = in ? ib.hi : T(0), il = in ? ib.lo : T(0);
    T u;
    if constexpr (use_hilo<T>()) u = fma(-ch, wn, fma(-cl, wn, y[t] * il));
    else u = -ch * wn;
    y[t] = fma(y[t], ih, u);
    wn = y[t];
  }
  const HiLo<T> pb0 = full ? HiLo<T>{p.qb[0][0], p.qb[1][0]} : HiLo<T>{T(0), T(0)};
  const T win = warp_chain_backward<T>(y[0], pb0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const HiLo<T> pbt = full ? HiLo<T>{p.qb[0][t], p.qb[1][t]} : HiLo<T>{T(0), T(0)};
    y[t] = fma2(pbt, win, y[t]);
  }
  if (lane == 0) y[0] = T(0);  // node 0: the wall
  // rank-one correction w = w' + kappa g w'_1 (w'_1: node 1, from its lane)
  const T w1 = (L >= 2) ? __shfl_sync(FULL, y[1 % L], 0) : __shfl_sync(FULL, y[0], 1);
#pragma unroll
  for (int t = 0; t < L; ++t) y[t] = fma2(HiLo<T>{kgh[t], kgl[t]}, w1, y[t]);
  // H update needs w at the next lane's first node (after the correction)
  T wnl = __shfl_down_sync(FULL, y[0], 1);
  if (lane == 31) wnl = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T wnext = (t + 1 < L) ? y[t + 1] : wnl;
    H[t] = fma(p.kd, wnext - y[t], H[t]);
  }
  e_update<T, L>(p, y, E);
  if (!ok) return;
  if (FULL_LINE || j0 + L <= N) {
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
  } else if (j0 < N) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t < N) {
        p.e_out[base + j0 + t] = E[t];
        p.h_out[base + j0 + t] = H[t];
      }
    }
  }
}

// Homogeneous media: the rank-one wall correction path when the host built
// it (p.wall_fix), else the table lanes.
template <typename T, int L>
__device__ __forceinline__ void row_solve_store_uniform(const PairParams<T>& p, long long line, T (&E)[L], T (&H)[L],
                                                        const T (&qn)[L], const T (&ibn)[L], const T (&ibl)[L]) {
  if (p.wall_fix) row_solve_store_wall<T, L>(p, line, E, H);
  else row_solve_store<T, L, false>(p, line, E, H, qn, ibn, ibl);
}

// Load this lane's segment of x line `line` (zeros past the line end).
// Segments never run past the padded row (the row pitch is >= 32*L).
template <typename T, int L, bool PER_NODE, bool FULL_LINE = false>
__device__ __forceinline__ void row_load(const PairParams<T>& p, long long line, T (&E)[L], T (&H)[L],
                                         T (&qn)[L], T (&ibn)[L], T (&ibl)[L]) {
  const int lane = threadIdx.x & 31;
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const int j0 = lane * L;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    qn[t] = T(0);
    ibn[t] = T(0);
    ibl[t] = T(0);
  }
  if ((FULL_LINE || j0 < p.N) && row_ok<T, L>(p, base)) {  // lanes wholly past the line end touch no memory
    load_seg<T, L>(p.e_in + base + j0, E);
    load_seg<T, L>(p.h_in + base + j0, H);
    if constexpr (PER_NODE) {
      load_seg<T, L>(p.nq + base + j0, qn);
      load_seg<T, L>(p.nib + base + j0, ibn);
      if constexpr (use_hilo<T>()) load_seg<T, L>(p.nibl + base + j0, ibl);
    }
  }
  if constexpr (!FULL_LINE) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t >= p.N) {
        E[t] = T(0);
        H[t] = T(0);
        qn[t] = T(0);
        ibn[t] = T(0);
        ibl[t] = T(0);
      }
    }
  }
}

// One warp per x line.  WALL: homogeneous media with the rank-one wall
// correction (p.wall_fix), a separate instantiation so that each path gets
// its own register allocation.  FULL_LINE (with WALL): lines of exactly 32 L
// cells, where every lane's nodes lie inside the line, so the end-of-line
// masks go (the same arithmetic on every node that the masked path keeps).
template <typename T, int L, bool PER_NODE, bool WALL = false, bool FULL_LINE = false>
__global__ void proc_rows_kernel(const PairParams<T> p) {
  const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= (long long)p.n_o * p.n_o2) return;  // whole warp leaves together
  T E[L], H[L], qn[L], ibn[L], ibl[L];
  row_load<T, L, PER_NODE, FULL_LINE>(p, line, E, H, qn, ibn, ibl);
  if constexpr (PER_NODE) row_solve_store<T, L, true>(p, line, E, H, qn, ibn, ibl);
  else if constexpr (WALL) row_solve_store_wall<T, L, FULL_LINE>(p, line, E, H);
  else row_solve_store<T, L, false>(p, line, E, H, qn, ibn, ibl);
}

// ---------------------------------------------------------------------------
// Lines along x, persistent, TMA-fed (homogeneous media, lines <= 256 cells)
// ---------------------------------------------------------------------------
// The one-warp-per-line kernel issues its loads only when a warp starts its
// line, so a warp spends a memory latency waiting before each solve.  Here
// a producer warp streams tiles of R consecutive rows (R x BN elements of E
// and of H, one 3-D TMA box each) into an NST-stage shared-memory ring, and
// R consumer warps each take one row of a tile: they copy their segments to
// registers, release the stage at once (an mbarrier arrival per warp, so the
// next tile's copy starts while they solve), then solve and store exactly as
// proc_rows_kernel does (bit-identical results).
struct RowTiles {
  int BN;         // elements per row box (>= N, a multiple of 8, <= 256)
  int tpp;        // tiles per plane: ceil(n_o / R)
  int n_tiles;    // tpp * n_o2
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Dynamic shared memory: [NST][E, H][R][BN] + 2 NST mbarriers (full, empty).
template <typename T, int L, int R, int NST, int MINB, bool WALL>
__global__ void __launch_bounds__((R + 1) * 32, MINB)
    proc_rows_tma_kernel(const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmH,
                         const PairParams<T> p, const RowTiles q) {
  static_assert(NST >= 2 && NST <= 4, "ring depth");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int stage_elems = R * q.BN;
  T* buf = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(buf + 2 * NST * stage_elems);
  uint64_t* empty = full + NST;
  const uint32_t stage_bytes = 2u * (uint32_t)stage_elems * (uint32_t)sizeof(T);

  if (threadIdx.x == 0) {
#pragma unroll
    for (int st = 0; st < NST; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], R);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == R) {
    // producer: one thread issues every copy of this block's tiles
    if (lane != 0) return;
    int k = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < q.n_tiles; tile += gridDim.x, ++k) {
      const int stage = k % NST;
      const uint32_t use = (uint32_t)(k / NST);
      if (use > 0 && !mbar_wait_bounded(&empty[stage], (use - 1) & 1u, kWaitLimitNs)) {
        atomicExch(p.err, 1);
        ok = false;
        break;
      }
      const int ko = p.o2_lo + tile / q.tpp;
      const int j0 = p.o_lo + (tile % q.tpp) * R;
      T* dE = buf + (2 * stage + 0) * stage_elems;
      T* dH = buf + (2 * stage + 1) * stage_elems;
      mbar_arrive_expect_tx(&full[stage], stage_bytes);
      tma_load_3d(dE, &tmE, &full[stage], 0, j0, ko);
      tma_load_3d(dH, &tmH, &full[stage], 0, j0, ko);
    }
    if (!ok) {
      // drain: the copies already issued land before the block may exit
      // (each wait bounded; a copy still outstanding after it is left in
      // flight, the host reports FDTD_ERR_TIMEOUT)
      for (int d = 1; d <= NST && k - d >= 0; ++d) {
        const int kk = k - d;
        mbar_wait_bounded(&full[kk % NST], (uint32_t)(kk / NST) & 1u, kWaitLimitNs);
      }
    }
    return;
  }

  // consumers: warp `warp` takes row `warp` of every tile
  int k = 0;
  for (int tile = blockIdx.x; tile < q.n_tiles; tile += gridDim.x, ++k) {
    const int stage = k % NST;
    const uint32_t use = (uint32_t)(k / NST);
    if (!mbar_wait_bounded(&full[stage], use & 1u, kWaitLimitNs)) {
      // give up: flag it; a second bounded wait lets this stage's copy land
      if (lane == 0) atomicExch(p.err, 1);
      mbar_wait_bounded(&full[stage], use & 1u, kWaitLimitNs);
      return;
    }
    const int kl = tile / q.tpp;
    const int jl = (tile % q.tpp) * R + warp;       // row within the pair's range
    const T* sE = buf + (2 * stage + 0) * stage_elems + warp * q.BN;
    const T* sH = buf + (2 * stage + 1) * stage_elems + warp * q.BN;
    const int j0 = lane * L;
    T E[L], H[L], qn[L], ibn[L], ibl[L];
#pragma unroll
    for (int t = 0; t < L; ++t) {
      qn[t] = T(0);
      ibn[t] = T(0);
      ibl[t] = T(0);
    }
    if (j0 + L <= q.BN) {
      load_seg<T, L>(sE + j0, E);
      load_seg<T, L>(sH + j0, H);
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        E[t] = T(0);
        H[t] = T(0);
      }
    }
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t >= p.N) {
        E[t] = T(0);
        H[t] = T(0);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[stage]);  // this warp is done with the stage
    if (jl < p.n_o) {
      const long long line = (long long)kl * p.n_o + jl;
      if constexpr (WALL) row_solve_store_wall<T, L>(p, line, E, H);
      else row_solve_store<T, L, false>(p, line, E, H, qn, ibn, ibl);
    }
  }
}

// ---------------------------------------------------------------------------
// Batched lines: many independent grids in one launch
// ---------------------------------------------------------------------------
// One launch covers the same pair of every grid of a batch.  y/z lines:
// tiles of LANES lines of one grid (tile table entry = (grid, x0, outer
// index)); a block holds G tiles, each on its own P * LANES threads (whole
// warps) with its own copy of its grid's parameters and its own carry
// buffers in shared memory, so that short lines still give blocks of a few
// hundred threads.  All tiles of a launch have the same segment count P and
// the same media kind (per-node or uniform), so every thread of a block
// passes the same barriers.  Spare tiles of the last block take part in the
// barriers with no active lane.
struct BatchTile {
  int grid, x0, o, pad;
};

template <typename T>
__host__ __device__ constexpr size_t batch_params_bytes(int G) {
  return ((sizeof(PairParams<T>) * (size_t)G + 15) / 16) * 16;
}

// One tile of LANES lines on the tpt = P * LANES threads of one slot (whole
// warps): tid is the thread's index in the slot, sh the slot's carry buffer,
// p its grid's parameters (shared memory).  have = false: a spare slot that
// passes the barriers of the solve with no active lane (no global access).
template <typename T, int LANES, int L>
__device__ __forceinline__ void strided_slot(const PairParams<T>& p, const BatchTile& tile, bool have, int tid,
                                             int tpt, T* sh) {
  const int P = tpt / LANES;
  const int lane = tid % LANES;
  const int s = tid / LANES;
  const int i = tile.x0 + lane;
  const int o = tile.o;
  const long long base = (long long)o * p.os + i;
  const bool active = have && (i >= p.lane_lo) && (i < p.lane_hi) && strided_line_ok(p, base);
  const int j0 = s * L;
  const int N = p.N;
  const long long ls = p.ls;
  const bool pn = p.nq != nullptr;

  T E[L], H[L], y[L], qn[L], ibn[L], ibl[L];
  HiLo<T> ib_prev = {T(0), T(0)};
  T hm1 = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    qn[t] = T(0);
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
        if (pn) {
          qn[t] = p.nq[at];
          ibn[t] = p.nib[at];
          if constexpr (use_hilo<T>()) ibl[t] = p.nibl[at];
        }
      }
    }
    if (j0 > 0 && j0 - 1 < N) {
      const long long at = base + (long long)(j0 - 1) * ls;
      hm1 = p.h_in[at];
      if (pn) {
        ib_prev.hi = p.nib[at];
        if constexpr (use_hilo<T>()) ib_prev.lo = p.nibl[at];
      }
    }
  }
  T win;
  if (pn) strided_solve<T, LANES, L, true>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, ib_prev, y, win, tid, tpt);
  else if (p.wall_fix) strided_solve_wall<T, LANES, L>(p, j0, s, P, lane, sh, E, H, hm1, y, win, tid, tpt);
  else strided_solve<T, LANES, L, false>(p, j0, s, P, lane, sh, E, H, hm1, qn, ibn, ibl, ib_prev, y, win, tid, tpt);
  if (active) strided_store<T, L>(p, base, j0, E, H, y, win);
}

// The tiles of one block: slots of tpt = P * LANES threads (whole warps) from
// thread 0 on, the first G of them holding tiles first .. first + G - 1;
// slots past those (or past the last tile), including a last slot with
// fewer than tpt threads, are spares that take part in the barriers with no
// active lane.  Shared memory: nslots parameter copies, then nslots carry
// buffers.
template <typename T, int LANES, int L>
__device__ __forceinline__ void strided_batch_block(const PairParams<T>* __restrict__ params,
                                                    const BatchTile* __restrict__ tiles, int ntiles, int G, int tpt,
                                                    int nslots, long long first, unsigned char* smem_raw) {
  const int sub = threadIdx.x / tpt;
  const int tid = threadIdx.x % tpt;
  const int P = tpt / LANES;
  const long long tix = first + sub;
  const bool have = sub < G && tix < ntiles;
  PairParams<T>* ps = reinterpret_cast<PairParams<T>*>(smem_raw);
  {
    // word copy of every slot's grid parameters (spare slots: the first tile's)
    static_assert(sizeof(PairParams<T>) % 4 == 0, "word copy");
    constexpr int W = (int)(sizeof(PairParams<T>) / 4);
    for (int k = threadIdx.x; k < nslots * W; k += blockDim.x) {
      const int sl = k / W;
      const long long tx = first + sl;
      const int grid = tiles[(sl < G && tx < ntiles) ? tx : first].grid;
      reinterpret_cast<int*>(ps + sl)[k % W] = reinterpret_cast<const int*>(params + grid)[k % W];
    }
  }
  __syncthreads();
  const BatchTile tile = tiles[have ? tix : first];
  T* sh = reinterpret_cast<T*>(smem_raw + batch_params_bytes<T>(nslots)) + (size_t)sub * 6 * chain_stride(P) * LANES;
  strided_slot<T, LANES, L>(ps[sub], tile, have, tid, tpt, sh);
}

template <typename T, int LANES, int L>
__global__ void proc_strided_batch_kernel(const PairParams<T>* __restrict__ params,
                                          const BatchTile* __restrict__ tiles, int ntiles, int G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  strided_batch_block<T, LANES, L>(params, tiles, ntiles, G, (int)blockDim.x / G, G, (long long)blockIdx.x * G,
                                   smem_raw);
}

// x lines of every grid of a group: one warp per line; line_start[g] is the
// first global line of the group's grid g (ascending, line_start[ngrids] =
// total).  All grids of a group share the segment length L of their tables.
template <typename T, int L>
__global__ void proc_rows_batch_kernel(const PairParams<T>* __restrict__ params,
                                       const long long* __restrict__ line_start, int ngrids) {
  const long long gline = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gline >= line_start[ngrids]) return;  // whole warp leaves together
  int lo = 0, hi = ngrids;                  // line_start[lo] <= gline < line_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (line_start[mid] <= gline) lo = mid;
    else hi = mid;
  }
  const PairParams<T>& p = params[lo];
  const long long line = gline - line_start[lo];
  T E[L], H[L], qn[L], ibn[L], ibl[L];
  if (p.nq != nullptr) {
    row_load<T, L, true>(p, line, E, H, qn, ibn, ibl);
    row_solve_store<T, L, true>(p, line, E, H, qn, ibn, ibl);
  } else {
    row_load<T, L, false>(p, line, E, H, qn, ibn, ibl);
    row_solve_store_uniform<T, L>(p, line, E, H, qn, ibn, ibl);
  }
}

// Carry chains across the LPL lanes of one line (a warp holds 32 / LPL
// lines; shuffles of width LPL keep the lines apart).
template <typename T, int LPL>
__device__ __forceinline__ T group_chain_forward(T a, HiLo<T> pm, int sl) {
  const unsigned FULL = 0xffffffffu;
  T pp = pm.hi;
#pragma unroll
  for (int d = 1; d < LPL; d <<= 1) {
    const T a_up = __shfl_up_sync(FULL, a, d, LPL);
    const T p_up = __shfl_up_sync(FULL, pp, d, LPL);
    if (sl >= d) {
      a = (d == 1) ? fma2(HiLo<T>{pp, pm.lo}, a_up, a) : fma(pp, a_up, a);
      pp = pp * p_up;
    }
  }
  const T yin = __shfl_up_sync(FULL, a, 1, LPL);
  return sl == 0 ? T(0) : yin;
}

template <typename T, int LPL>
__device__ __forceinline__ T group_chain_backward(T b, HiLo<T> pm, int sl) {
  const unsigned FULL = 0xffffffffu;
  T qq = pm.hi;
#pragma unroll
  for (int d = 1; d < LPL; d <<= 1) {
    const T b_dn = __shfl_down_sync(FULL, b, d, LPL);
    const T q_dn = __shfl_down_sync(FULL, qq, d, LPL);
    if (sl + d < LPL) {
      b = (d == 1) ? fma2(HiLo<T>{qq, pm.lo}, b_dn, b) : fma(qq, b_dn, b);
      qq = qq * q_dn;
    }
  }
  const T win = __shfl_down_sync(FULL, b, 1, LPL);
  return sl == LPL - 1 ? T(0) : win;
}

// x lines of uniform media, LPL lanes per line (32 / LPL lines per warp) and
// L nodes per lane, for FP64 fields, whose FP64 pipe bounds the solve.  Every
// lane reads its coefficients from the tables (MODE 0): a warp spans whole
// lines, so lanes at the walls and lanes in the converged interior would
// otherwise take different branches, and the warp would issue the FP64
// arithmetic of both.  The carry chains take log2(LPL) shuffle steps.  The
// coefficient tables are built for this L.
template <typename T, int L, int LPL>
__global__ void proc_rows_lpl_kernel(const PairParams<T> p) {
  constexpr int LPW = 32 / LPL;  // lines per warp
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int sl = lane % LPL;
  const long long n = (long long)p.n_o * p.n_o2;
  const long long gwarp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gwarp * LPW >= n) return;  // whole warp leaves together
  const long long gline = gwarp * LPW + lane / LPL;
  const bool in_grid = gline < n;
  const long long line = in_grid ? gline : n - 1;
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const bool ok = in_grid && row_ok<T, L>(p, base);
  const int j0 = sl * L;
  const int N = p.N;

  T E[L], H[L], qn[L], ibn[L], ibl[L], y[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    qn[t] = T(0);
    ibn[t] = T(0);
    ibl[t] = T(0);
  }
  if (ok && j0 < N) {
    load_seg<T, L>(p.e_in + base + j0, E);
    load_seg<T, L>(p.h_in + base + j0, H);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t >= N) {
        E[t] = T(0);
        H[t] = T(0);
      }
    }
  }
  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1, LPL);
  if (sl == 0) hm1 = T(0);
  const HiLo<T> ib_prev = {T(0), T(0)};
  const HiLo<T> pf = phase_forward<T, L, 0>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
  const T yin = group_chain_forward<T, LPL>(y[L - 1], pf, sl);
  const HiLo<T> pb = phase_backward<T, L, 0>(p, j0, yin, ibn, ibl, ib_prev, y);
  const T win = group_chain_backward<T, LPL>(y[0], pb, sl);
  phase_fix<T, L, 0>(p, j0, win, ibn, ibl, y);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T wnext = (t + 1 < L) ? y[t + 1] : win;
    H[t] = fma(p.kd, wnext - y[t], H[t]);
  }
  e_update<T, L>(p, y, E);
  if (!ok) return;
  if (j0 + L <= N) {
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
  } else if (j0 < N) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      if (j0 + t < N) {
        p.e_out[base + j0 + t] = E[t];
        p.h_out[base + j0 + t] = H[t];
      }
    }
  }
}

// x lines of per-node grids in a batch, LPL lanes per line and L nodes per
// lane (LPL * L >= N): short lines share a warp so that every lane still
// streams L nodes of each array.  line_start as for proc_rows_batch_kernel.
// Whole segments inside the line move as 16-byte vectors; the segment
// holding the line end is read and written element by element, so no
// access leaves the line.  Lines past the last one take part in the
// shuffles without touching memory.
template <typename T, int L, int LPL>
__device__ __forceinline__ void rows_batch_pn_warp(const PairParams<T>* __restrict__ params,
                                                   const long long* __restrict__ line_start, int ngrids,
                                                   long long gwarp) {
  constexpr int LPW = 32 / LPL;  // lines per warp
  const int lane = threadIdx.x & 31;
  const int sl = lane % LPL;
  const long long total = line_start[ngrids];
  if (gwarp * LPW >= total) return;  // whole warp leaves together
  const long long gline = gwarp * LPW + lane / LPL;
  const bool in_batch = gline < total;
  const long long gl = in_batch ? gline : total - 1;
  int lo = 0, hi = ngrids;  // line_start[lo] <= gl < line_start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (line_start[mid] <= gl) lo = mid;
    else hi = mid;
  }
  const PairParams<T>& p = params[lo];
  const long long line = gl - line_start[lo];
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const int j0 = sl * L;
  const int N = p.N;
  const bool valid = in_batch && FDTD_IN_RANGE(base, base + N, p.n_elem);
  const bool full = j0 + L <= N;

  T E[L], H[L], qn[L], ibn[L], ibl[L], y[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = T(0);
    H[t] = T(0);
    qn[t] = T(0);
    ibn[t] = T(0);
    ibl[t] = T(0);
  }
  if (valid) {
    if (full) {
      load_seg<T, L>(p.e_in + base + j0, E);
      load_seg<T, L>(p.h_in + base + j0, H);
      load_seg<T, L>(p.nq + base + j0, qn);
      load_seg<T, L>(p.nib + base + j0, ibn);
      if constexpr (use_hilo<T>()) load_seg<T, L>(p.nibl + base + j0, ibl);
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        if (j0 + t < N) {
          const long long at = base + j0 + t;
          E[t] = p.e_in[at];
          H[t] = p.h_in[at];
          qn[t] = p.nq[at];
          ibn[t] = p.nib[at];
          if constexpr (use_hilo<T>()) ibl[t] = p.nibl[at];
        }
      }
    }
  }
  const unsigned FULL = 0xffffffffu;
  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1, LPL);
  HiLo<T> ib_prev = {__shfl_up_sync(FULL, ibn[L - 1], 1, LPL), T(0)};
  if constexpr (use_hilo<T>()) ib_prev.lo = __shfl_up_sync(FULL, ibl[L - 1], 1, LPL);
  if (sl == 0) {
    hm1 = T(0);
    ib_prev = {T(0), T(0)};
  }
  const HiLo<T> pf = phase_forward<T, L, 2>(p, j0, E, H, hm1, qn, ibn, ibl, ib_prev, y);
  const T yin = group_chain_forward<T, LPL>(y[L - 1], pf, sl);
  const HiLo<T> pb = phase_backward<T, L, 2>(p, j0, yin, ibn, ibl, ib_prev, y);
  const T win = group_chain_backward<T, LPL>(y[0], pb, sl);
  phase_fix<T, L, 2>(p, j0, win, ibn, ibl, y);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T wnext = (t + 1 < L) ? y[t + 1] : win;
    H[t] = fma(p.kd, wnext - y[t], H[t]);
  }
  e_update<T, L>(p, y, E);
  if (!valid) return;
  if (full) {
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

template <typename T, int L, int LPL>
__global__ void proc_rows_batch_pn_kernel(const PairParams<T>* __restrict__ params,
                                          const long long* __restrict__ line_start, int ngrids) {
  rows_batch_pn_warp<T, L, LPL>(params, line_start, ngrids,
                                (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------------------
// A whole procedure of a batch in one persistent launch
// ---------------------------------------------------------------------------
// The work of one procedure (its three pairs on every grid) is a list of
// items, each a block's worth of work: y/z tiles of per-node grids packed
// into slots of P * LANES threads (tiles of different segment counts P side
// by side; a last spare slot takes the threads left over), or blockDim / 32
// warps of an x group of per-node grids (LPL lanes per line).  Every block
// takes the next item from a counter (zeroed before the launch) until the
// list is exhausted; every thread of the block belongs to exactly one slot
// of a y/z item and runs the same solve code, so all pass the same barriers,
// and the loop ends after at most one pass over the list.
struct BatchWork {
  int group;        // x items: the x group; y/z items: -1
  int nslots;       // y/z items: slots of the item
  long long first;  // x: first warp; y/z: first slot in the slot list
};

struct BatchSlot {
  int group;  // y/z group of the tile (spare slot: that of slot 0)
  int tile;   // tile index in the group; -1: the spare slot
  int toff;   // first thread of the slot (slots ascend)
  int tpt;    // threads of the slot: P * LANES
  int coff;   // offset of its carry buffer (elements of T) after the parameter copies
  int pad;
};

template <typename T>
struct BatchGroupRef {
  const PairParams<T>* params;  // [ngrids]
  const void* index;            // y/z: BatchTile[nitems]; x: line_start[ngrids + 1]
  long long nitems;             // y/z: tiles; x: lines
  int ngrids;
  int kind;                     // 0 y/z tiles, 1 x lines of per-node grids
  int P, G, lpl, pad;           // y/z: segments and tiles per item; x: lanes per line
};

template <typename T, int LANES, int L>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && L == 8) ? 3 : 2) proc_batch_persistent_kernel(const BatchGroupRef<T>* __restrict__ groups,
                                                                     const BatchWork* __restrict__ work,
                                                                     const BatchSlot* __restrict__ slots, int nwork,
                                                                     int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int w = s_next;
    if (w >= nwork) break;  // the same value in every thread of the block
    const BatchWork item = work[w];
    if (item.group < 0) {
      const BatchSlot* sl = slots + item.first;
      const int ns = item.nslots;
      int my = 0;
      for (int k = 1; k < ns; ++k)
        if ((int)threadIdx.x >= sl[k].toff) my = k;
      PairParams<T>* ps = reinterpret_cast<PairParams<T>*>(smem_raw);
      {
        // word copy of every slot's grid parameters (the spare: slot 0's)
        constexpr int W = (int)(sizeof(PairParams<T>) / 4);
        for (int k = threadIdx.x; k < ns * W; k += blockDim.x) {
          const int q = k / W;
          const BatchSlot& b = sl[q].tile >= 0 ? sl[q] : sl[0];
          const BatchGroupRef<T>& gq = groups[b.group];
          const int grid = static_cast<const BatchTile*>(gq.index)[b.tile].grid;
          reinterpret_cast<int*>(ps + q)[k % W] = reinterpret_cast<const int*>(gq.params + grid)[k % W];
        }
      }
      __syncthreads();
      const BatchSlot me = sl[my];
      const bool have = me.tile >= 0;
      const BatchSlot& src = have ? me : sl[0];
      const BatchTile tile = static_cast<const BatchTile*>(groups[src.group].index)[src.tile];
      T* sh = reinterpret_cast<T*>(smem_raw + batch_params_bytes<T>(ns)) + me.coff;
      strided_slot<T, LANES, L>(ps[my], tile, have, (int)threadIdx.x - me.toff, me.tpt, sh);
    } else {
      const BatchGroupRef<T> g = groups[item.group];
      const long long gwarp = item.first + (threadIdx.x >> 5);
      const long long* ls = static_cast<const long long*>(g.index);
      if (g.lpl == 8) rows_batch_pn_warp<T, 8, 8>(g.params, ls, g.ngrids, gwarp);
      else if (g.lpl == 16) rows_batch_pn_warp<T, 8, 16>(g.params, ls, g.ngrids, gwarp);
      else rows_batch_pn_warp<T, 8, 32>(g.params, ls, g.ngrids, gwarp);
    }
    __syncthreads();  // the next item reuses the shared memory and s_next
  }
}

// ---------------------------------------------------------------------------
// General media: per-node eps and mu.  The scaled symmetric rows of the
// per-node form keep their shape, but each face has its own off-diagonal
// off_f = -|ks| |kd_f| / 2 and H coupling kd_f: m_j = off_{j-1} / beta_{j-1},
// c_j = off_j / beta_j.  offh/offl[t]: face j0 + t; off_prev: face j0 - 1.
// ---------------------------------------------------------------------------
template <typename T, int L>
__device__ __forceinline__ HiLo<T> gm_m(int t, const T (&ibn)[L], const T (&ibl)[L], HiLo<T> ib_prev,
                                        const T (&offh)[L], const T (&offl)[L], HiLo<T> off_prev) {
  if (t == 0) return dd_mul(off_prev, ib_prev);
  return dd_mul(HiLo<T>{offh[t - 1], offl[t - 1]}, HiLo<T>{ibn[t - 1], ibl[t - 1]});
}
template <typename T, int L>
__device__ __forceinline__ HiLo<T> gm_c(int t, const T (&ibn)[L], const T (&ibl)[L], const T (&offh)[L],
                                        const T (&offl)[L]) {
  return dd_mul(HiLo<T>{offh[t], offl[t]}, HiLo<T>{ibn[t], ibl[t]});
}

template <typename T, int L>
__device__ __forceinline__ HiLo<T> gm_forward(const PairParams<T>& p, const T (&E)[L], const T (&H)[L], T hm1,
                                              const T (&qn)[L], const T (&ibn)[L], const T (&ibl)[L],
                                              HiLo<T> ib_prev, const T (&offh)[L], const T (&offl)[L],
                                              HiLo<T> off_prev, T (&y)[L]) {
  T pf = T(1), hprev = hm1;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T r = fma(qn[t], E[t], p.ks * (H[t] - hprev));
    hprev = H[t];
    const HiLo<T> m = gm_m<T, L>(t, ibn, ibl, ib_prev, offh, offl, off_prev);
    y[t] = (t == 0) ? r : fma2(HiLo<T>{-m.hi, -m.lo}, y[t - 1], r);
    pf *= -m.hi;
  }
  return {pf, T(0)};
}

template <typename T, int L>
__device__ __forceinline__ HiLo<T> gm_backward(T yin, const T (&ibn)[L], const T (&ibl)[L], HiLo<T> ib_prev,
                                               const T (&offh)[L], const T (&offl)[L], HiLo<T> off_prev,
                                               T (&y)[L]) {
  T q = T(1);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    q *= -gm_m<T, L>(t, ibn, ibl, ib_prev, offh, offl, off_prev).hi;
    y[t] = fma(q, yin, y[t]);
  }
  T pb = T(1), wn = T(0);
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    const HiLo<T> c = gm_c<T, L>(t, ibn, ibl, offh, offl);
    T u;
    if constexpr (use_hilo<T>()) u = fma(-c.hi, wn, fma(-c.lo, wn, y[t] * ibl[t]));
    else u = -c.hi * wn;
    y[t] = fma(y[t], ibn[t], u);
    wn = y[t];
    pb *= -c.hi;
  }
  return {pb, T(0)};
}

template <typename T, int L>
__device__ __forceinline__ void gm_fix(T win, const T (&ibn)[L], const T (&ibl)[L], const T (&offh)[L],
                                       const T (&offl)[L], T (&y)[L]) {
  T q = T(1);
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    q *= -gm_c<T, L>(t, ibn, ibl, offh, offl).hi;
    y[t] = fma(q, win, y[t]);
  }
}

// Lines along y or z in general media (one block per LANES lines, loads
// straight from HBM).
template <typename T, int LANES, int L>
__global__ void proc_strided_gm_kernel(const PairParams<T> p) {
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

  T E[L], H[L], y[L], qn[L], ibn[L], ibl[L], offh[L], offl[L], kd[L];
  HiLo<T> ib_prev = {T(0), T(0)}, off_prev = {T(0), T(0)};
  T hm1 = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = H[t] = qn[t] = ibn[t] = ibl[t] = offh[t] = offl[t] = kd[t] = T(0);
  }
  if (active) {
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int j = j0 + t;
      if (j < N) {
        const long long at = base + (long long)j * ls;
        E[t] = p.e_in[at];
        H[t] = p.h_in[at];
        qn[t] = p.nq[at];
        ibn[t] = p.nib[at];
        offh[t] = p.noffh[at];
        kd[t] = p.nkd[at];
        if constexpr (use_hilo<T>()) {
          ibl[t] = p.nibl[at];
          offl[t] = p.noffl[at];
        }
      }
    }
    if (j0 > 0 && j0 - 1 < N) {
      const long long at = base + (long long)(j0 - 1) * ls;
      hm1 = p.h_in[at];
      ib_prev.hi = p.nib[at];
      off_prev.hi = p.noffh[at];
      if constexpr (use_hilo<T>()) {
        ib_prev.lo = p.nibl[at];
        off_prev.lo = p.noffl[at];
      }
    }
  }
  const int PW = pow2_at_least(P);
  const HiLo<T> pf = gm_forward<T, L>(p, E, H, hm1, qn, ibn, ibl, ib_prev, offh, offl, off_prev, y);
  const T yin = block_chain_forward<T, LANES>(sh, P, PW, s, lane, y[L - 1], pf, (int)threadIdx.x, (int)blockDim.x);
  const HiLo<T> pb = gm_backward<T, L>(yin, ibn, ibl, ib_prev, offh, offl, off_prev, y);
  const T win = block_chain_backward<T, LANES>(sh, P, PW, s, lane, y[0], pb, (int)threadIdx.x, (int)blockDim.x);
  gm_fix<T, L>(win, ibn, ibl, offh, offl, y);
  if (!active) return;
  T En[L];
  e_next<T, L>(p, y, E, En);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const int j = j0 + t;
    if (j < N) {
      const long long at = base + (long long)j * ls;
      const T wnext = (t + 1 < L) ? y[t + 1] : win;
      p.e_out[at] = En[t];
      p.h_out[at] = fma(p.kd_scale * kd[t], wnext - y[t], H[t]);
    }
  }
}

// x lines in general media: one warp per line, L = nodes per lane (32 L >= N;
// the row pitch is >= 32 L, so whole-segment loads stay inside the row).
template <typename T, int L>
__global__ void proc_rows_gm_kernel(const PairParams<T> p) {
  const unsigned FULL = 0xffffffffu;
  const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= (long long)p.n_o * p.n_o2) return;  // whole warp leaves together
  const int lane = threadIdx.x & 31;
  const int jo = p.o_lo + (int)(line % p.n_o);
  const int ko = p.o2_lo + (int)(line / p.n_o);
  const long long base = (long long)ko * p.os2 + (long long)jo * p.os;
  const bool ok = row_ok<T, L>(p, base);
  const int j0 = lane * L;
  const int N = p.N;
  T E[L], H[L], y[L], qn[L], ibn[L], ibl[L], offh[L], offl[L], kd[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    E[t] = H[t] = qn[t] = ibn[t] = ibl[t] = offh[t] = offl[t] = kd[t] = T(0);
  }
  if (j0 < N && ok) {
    load_seg<T, L>(p.e_in + base + j0, E);
    load_seg<T, L>(p.h_in + base + j0, H);
    load_seg<T, L>(p.nq + base + j0, qn);
    load_seg<T, L>(p.nib + base + j0, ibn);
    load_seg<T, L>(p.noffh + base + j0, offh);
    load_seg<T, L>(p.nkd + base + j0, kd);
    if constexpr (use_hilo<T>()) {
      load_seg<T, L>(p.nibl + base + j0, ibl);
      load_seg<T, L>(p.noffl + base + j0, offl);
    }
  }
#pragma unroll
  for (int t = 0; t < L; ++t) {
    if (j0 + t >= N) E[t] = H[t] = qn[t] = ibn[t] = ibl[t] = offh[t] = offl[t] = kd[t] = T(0);
  }
  T hm1 = __shfl_up_sync(FULL, H[L - 1], 1);
  HiLo<T> ib_prev = {__shfl_up_sync(FULL, ibn[L - 1], 1), __shfl_up_sync(FULL, ibl[L - 1], 1)};
  HiLo<T> off_prev = {__shfl_up_sync(FULL, offh[L - 1], 1), __shfl_up_sync(FULL, offl[L - 1], 1)};
  if (lane == 0) {
    hm1 = T(0);
    ib_prev = {T(0), T(0)};
    off_prev = {T(0), T(0)};
  }
  const HiLo<T> pf = gm_forward<T, L>(p, E, H, hm1, qn, ibn, ibl, ib_prev, offh, offl, off_prev, y);
  const T yin = warp_chain_forward<T>(y[L - 1], pf);
  const HiLo<T> pb = gm_backward<T, L>(yin, ibn, ibl, ib_prev, offh, offl, off_prev, y);
  const T win = warp_chain_backward<T>(y[0], pb);
  gm_fix<T, L>(win, ibn, ibl, offh, offl, y);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const T wnext = (t + 1 < L) ? y[t + 1] : win;
    H[t] = fma(p.kd_scale * kd[t], wnext - y[t], H[t]);
  }
  e_update<T, L>(p, y, E);
  if (!ok) return;
  if (j0 + L <= N) {
    store_seg<T, L>(p.e_out + base + j0, E);
    store_seg<T, L>(p.h_out + base + j0, H);
  } else if (j0 < N) {
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
