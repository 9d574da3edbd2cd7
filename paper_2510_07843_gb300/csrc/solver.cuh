// Per-RE FP32 LMMSE solve, one thread per resource element.
//
// Given the Gram matrix A = H^H H + s2 I (Hermitian positive definite, supplied entry by entry
// through a functor so that callers can build it on the fly) and the matched filter b = H^H y,
// computes x = A^-1 b and d_k = (A^-1)_kk. The paper's LMMSE block (Sec. IV, Fig. 3) factors
// the matrix to invert and runs forward/backward substitution; here A is factored by Cholesky
// A = L L^H (it is Hermitian positive definite), x by the two triangular solves, and the diagonal
// of the inverse by the column norms of L^-1, since (A^-1)_kk = sum_i |(L^-1)_ik|^2.
//
// Up to 8 layers the packed lower triangle lives in registers. For 9..16 layers the matrix is
// split into 8x8 blocks, A = [A11 A12; A21 A22]:
//   L11 = chol(A11), M = L11^-1, L21 = A21 M^H, S = A22 - L21 L21^H, L22 = chol(S), N = L22^-1,
//   L^-1 = [M 0; -N T  N] with T = L21 M,
// so z = L^-1 b = [M b1; N (b2 - L21 z1)], x = L^-H z = [M^H z1 - T^H x2; N^H z2], and the
// column norms of L^-1 give d: block 2 from N, block 1 from M and N T.
#pragma once

#include "common.cuh"

namespace phy {

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Cholesky in place on a packed lower triangle (left-looking). rinv[j] = 1 / L_jj; the diagonal
// entries of `a` are left holding the pivots L_jj^2. Returns false on a non-positive or
// non-finite pivot; fin turns false on a non-finite one.
template <int N>
__device__ __forceinline__ bool chol_packed(cf (&a)[N * (N + 1) / 2], float (&rinv)[N],
                                            float& pmin, float& pmax, bool& fin) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float d = a[tri(j, j)].x;
#pragma unroll
    for (int k = 0; k < j; ++k) d -= cabs2(a[tri(j, k)]);
    // a non-finite pivot after an earlier failed one is a consequence, not bad input
    if (ok) fin = fin && isfinite(d);
    ok = ok && (d > 0.f) && (d < 3.0e38f);
    pmin = fminf(pmin, d);
    pmax = fmaxf(pmax, d);
    a[tri(j, j)] = mk(d, 0.f);
    const float r = rsqrtf(d);
    rinv[j] = r;
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      cf s = a[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s = cfms_cjb(a[tri(i, k)], a[tri(j, k)], s);
      a[tri(i, j)] = r * s;
    }
  }
  return ok;
}

// z = L^-1 b (forward substitution) for the factor produced by chol_packed.
template <int N>
__device__ __forceinline__ void fwd_packed(const cf (&a)[N * (N + 1) / 2], const float (&rinv)[N],
                                           const cf (&b)[N], cf (&z)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    cf s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = cfms(a[tri(i, k)], z[k], s);
    z[i] = rinv[i] * s;
  }
}

// x = L^-H z (backward substitution).
template <int N>
__device__ __forceinline__ void bwd_packed(const cf (&a)[N * (N + 1) / 2], const float (&rinv)[N],
                                           const cf (&z)[N], cf (&x)[N]) {
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    cf s = z[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) {
      // s -= conj(L_ki) x_k
      const cf l = a[tri(k, i)];
      s.x = fmaf(-l.x, x[k].x, s.x);
      s.x = fmaf(-l.y, x[k].y, s.x);
      s.y = fmaf(-l.x, x[k].y, s.y);
      s.y = fmaf(l.y, x[k].x, s.y);
    }
    x[i] = rinv[i] * s;
  }
}

// Overwrite the strictly-lower part of the factor with that of L^-1; its diagonal is rinv.
// Columns left to right, rows top to bottom: entry (i, c) of the inverse needs row i of L at
// columns >= c (still intact) and rows < i of the inverse's column c (already written).
template <int N>
__device__ __forceinline__ void inv_packed(cf (&a)[N * (N + 1) / 2], const float (&rinv)[N]) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
#pragma unroll
    for (int i = c + 1; i < N; ++i) {
      // (L^-1)_ic = -(L_ic (L^-1)_cc + sum_{c<m<i} L_im (L^-1)_mc) / L_ii
      cf s = rinv[c] * a[tri(i, c)];
#pragma unroll
      for (int m = c + 1; m < i; ++m) s = cfma(a[tri(i, m)], a[tri(m, c)], s);
      a[tri(i, c)] = (-rinv[i]) * s;
    }
  }
}

// Column norms of the lower-triangular inverse stored by inv_packed.
template <int N>
__device__ __forceinline__ void colnorm_inv(const cf (&a)[N * (N + 1) / 2], const float (&rinv)[N],
                                            float (&d)[N]) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
    float s = rinv[c] * rinv[c];
#pragma unroll
    for (int i = c + 1; i < N; ++i) s += cabs2(a[tri(i, c)]);
    d[c] = s;
  }
}

struct SolveInfo {
  bool ok;    // every pivot positive and finite
  bool fin;   // every pivot finite (false points at non-finite input)
  float pmin, pmax;
};

// Up to 8 layers: everything in registers.
template <int N, class GetA>
__device__ __forceinline__ SolveInfo solve_small(GetA getA, const cf (&b)[N], cf (&x)[N],
                                                 float (&d)[N]) {
  cf a[N * (N + 1) / 2];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) a[tri(i, j)] = getA(i, j);
  float rinv[N];
  SolveInfo si{true, true, 3.0e38f, 0.f};
  si.ok = chol_packed<N>(a, rinv, si.pmin, si.pmax, si.fin);
  cf z[N];
  fwd_packed<N>(a, rinv, b, z);
  bwd_packed<N>(a, rinv, z, x);
  inv_packed<N>(a, rinv);
  colnorm_inv<N>(a, rinv, d);
  return si;
}

// 9..16 layers: two 8x8 blocks. The thread's 8x8 L21 (later overwritten by T = L21 M) lives
// off registers in `rows`, which stores and loads it a row or a column at a time
// (st_row(i, r) / ld_row(i, r) / ld_col(c, col), then sync_st() once a pass of stores must be
// visible to the next pass's loads), and an 8-vector lives in the thread-private scratch `vs`
// (ld(e) / st(e, v), e < 8). M and the Schur complement are in registers, but never both
// factored at once: everything that needs M (L21, T, M^H z1, the column norms of M) is done
// before the Schur complement is factored, so M is dead by then and x1 comes from T as
// x1 = M^H z1 - T^H x2. The large repeated pieces (rows of L21 and T, the Schur update, the
// columns of N T) are runtime loops over small unrolled bodies: the kernel's code then fits the
// instruction cache, which the fully unrolled form did not. Every thread of a warp must take
// part (the tensor-memory form of `rows` is warp-collective).
constexpr int kScrL21 = 0, kScrV = 64, kScrSlots = 72;

// rowA(l, row) fills row[k] = A(l, k), k = 0..7, for a row l >= 8 known only at run time (the
// runtime-row form of getA, for the rolled L21 loop).
template <class GetA, class RowA, class Vec, class Rows>
__device__ __forceinline__ SolveInfo solve16(GetA getA, RowA rowA, Vec vs, Rows rows,
                                             const cf (&b)[16], cf (&x)[16], float (&d)[16]) {
  constexpr int B = 8;
  SolveInfo si{true, true, 3.0e38f, 0.f};
  // ---- block 1: L11, z1 = L11^-1 b1, M = L11^-1
  cf m[B * (B + 1) / 2];
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) m[tri(i, j)] = getA(i, j);
  float r1[B];
  si.ok = chol_packed<B>(m, r1, si.pmin, si.pmax, si.fin);
  cf b1[B], z1[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    b1[i] = b[i];
    vs.st(i, b[B + i]);
  }
  fwd_packed<B>(m, r1, b1, z1);
  inv_packed<B>(m, r1);
  auto M = [&](int i, int j) -> cf { return (i == j) ? mk(r1[i], 0.f) : m[tri(i, j)]; };
  // ---- L21 = A21 M^H row by row; v = b2 - L21 z1
#pragma unroll 1
  for (int i = 0; i < B; ++i) {
    cf row[B], l21[B];
    rowA(B + i, row);
    cf acc = vs.ld(i), acc2 = mk(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      cf l = mk(0.f, 0.f);
#pragma unroll
      for (int k = 0; k <= j; ++k) l = cfma_cj(M(j, k), row[k], l);  // row[k] conj(M[j][k])
      l21[j] = l;
      if (j & 1)
        acc2 = cfms(l, z1[j], acc2);
      else
        acc = cfms(l, z1[j], acc);
    }
    rows.st_row(i, l21);
    vs.st(i, acc + acc2);
  }
  rows.sync_st();
  // ---- w = M^H z1, and the column norms of M (the first part of d for block 1)
  cf w[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    cf acc = mk(0.f, 0.f);
    float s1 = r1[i] * r1[i];
#pragma unroll
    for (int k = i; k < B; ++k) acc = cfma_cj(M(k, i), z1[k], acc);
#pragma unroll
    for (int k = i + 1; k < B; ++k) s1 += cabs2(M(k, i));
    w[i] = acc;
    d[i] = s1;
  }
  // ---- S = A22 - L21 L21^H
  cf s[B * (B + 1) / 2];
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) s[tri(i, j)] = getA(B + i, B + j);
#pragma unroll 1
  for (int c = 0; c < B; ++c) {
    cf col[B];
    rows.ld_col(c, col);
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) s[tri(i, j)] = cfms_cjb(col[i], col[j], s[tri(i, j)]);
  }
  // ---- T = L21 M, row i of T from row i of L21, written over it (M is dead after this)
#pragma unroll 1
  for (int i = 0; i < B; ++i) {
    cf row[B], trow[B];
    rows.ld_row(i, row);
#pragma unroll
    for (int c = 0; c < B; ++c) {
      cf acc = mk(0.f, 0.f);
#pragma unroll
      for (int k = c; k < B; ++k) acc = cfma(row[k], M(k, c), acc);
      trow[c] = acc;
    }
    rows.st_row(i, trow);
  }
  rows.sync_st();
  // ---- block 2: L22 = chol(S), z2 = L22^-1 v, x2 = L22^-H z2, N = L22^-1
  float r2[B];
  si.ok = chol_packed<B>(s, r2, si.pmin, si.pmax, si.fin) && si.ok;
  cf v[B], z2[B], x2[B];
#pragma unroll
  for (int i = 0; i < B; ++i) v[i] = vs.ld(i);
  fwd_packed<B>(s, r2, v, z2);
  bwd_packed<B>(s, r2, z2, x2);
  inv_packed<B>(s, r2);
  auto Nn = [&](int i, int j) -> cf { return (i == j) ? mk(r2[i], 0.f) : s[tri(i, j)]; };
  // ---- x1 = w - T^H x2
#pragma unroll
  for (int i = 0; i < B; ++i) {
    cf row[B];
    rows.ld_row(i, row);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      // w_j -= conj(T_ij) x2_i
      const cf t = row[j];
      w[j].x = fmaf(-t.x, x2[i].x, w[j].x);
      w[j].x = fmaf(-t.y, x2[i].y, w[j].x);
      w[j].y = fmaf(-t.x, x2[i].y, w[j].y);
      w[j].y = fmaf(t.y, x2[i].x, w[j].y);
    }
  }
#pragma unroll
  for (int i = 0; i < B; ++i) {
    x[i] = w[i];
    x[B + i] = x2[i];
  }
  // ---- diagonal of A^-1. Block 2: column norms of N. Block 1: those of M (above) plus those
  // of N T.
#pragma unroll
  for (int c = 0; c < B; ++c) {
    float s2 = 0.f;
#pragma unroll
    for (int i = c; i < B; ++i) s2 += cabs2(Nn(i, c));
    d[B + c] = s2;
  }
#pragma unroll 1
  for (int c = 0; c < B; ++c) {
    cf t[B];
    rows.ld_col(c, t);
    float acc2 = 0.f;
#pragma unroll
    for (int i = 0; i < B; ++i) {  // (N t)_i
      cf p = mk(0.f, 0.f);
#pragma unroll
      for (int k = 0; k <= i; ++k) p = cfma(Nn(i, k), t[k], p);
      acc2 += cabs2(p);
    }
#pragma unroll
    for (int cc = 0; cc < B; ++cc)  // d[c] += acc2 without indexing registers at run time
      if (cc == c) d[cc] += acc2;
  }
  return si;
}

}  // namespace phy
