// Solves with the tree-sparse factor M = L^T D L that frax_crba returns
// (packed lower triangle: D on the diagonal, L below). L_kj is nonzero only
// for dofs j on the path from dof k to the root, so both substitutions walk
// dof-parent chains: O(nv * depth) per right-hand side.
#pragma once
#include "dyn.cuh"

namespace frax {

// x = M^-1 b: L^T y = b by back substitution (each dof, once final, is
// subtracted from its ancestors), then L x = D^-1 y by forward substitution.
template <class T, class Img, class C, class Rhs, class Out>
FD void ltdl_solve_one(const Img& M, const float* __restrict__ LD, const Rhs& b_at, const Out& x_to,
                       const C& col) {
  const int nv = T::kFree ? T::nb(M) + 5 : T::nb(M);
  float y[T::NVMAX];
#pragma unroll(T::kStatic ? T::NVMAX : 1)
  for (int k = 0; k < T::NVMAX; ++k)
    if (k < nv) y[k] = b_at(k);
#pragma unroll(T::kStatic ? T::NVMAX : 1)
  for (int k = T::NVMAX - 1; k >= 0; --k) {
    if (k >= nv) continue;
    const float yk = y[k];
    int j = T::dparent(M, k);
#pragma unroll(T::kStatic ? T::NVMAX : 1)
    for (int step = 0; step < T::NVMAX; ++step) {
      if (j < 0) break;
      y[j] = fmaf(-col.in(LD, MSink::tri(k, j)), yk, y[j]);
      j = T::dparent(M, j);
    }
  }
#pragma unroll(T::kStatic ? T::NVMAX : 1)
  for (int k = 0; k < T::NVMAX; ++k) {
    if (k >= nv) break;
    float x = y[k] * rcp(col.in(LD, MSink::tri(k, k)));
    int j = T::dparent(M, k);
#pragma unroll(T::kStatic ? T::NVMAX : 1)
    for (int step = 0; step < T::NVMAX; ++step) {
      if (j < 0) break;
      x = fmaf(-col.in(LD, MSink::tri(k, j)), y[j], x);
      j = T::dparent(M, j);
    }
    y[k] = x;  // ancestors j < k already hold x_j
    x_to(k, x);
  }
}

template <class C>
struct VecIn {
  const float* p;
  C col;
  FD float operator()(int k) const { return col.in(p, k); }
};
template <class C>
struct VecOut {
  float* p;
  C col;
  FD void operator()(int k, float v) const { col.out(p, k, v); }
};
// unit vector e_c
struct UnitIn {
  int c;
  FD float operator()(int k) const { return k == c ? 1.f : 0.f; }
};
// column c of a row-major nv x nv matrix
template <class C>
struct ColOut {
  float* p;
  int c, nv;
  C col;
  FD void operator()(int k, float v) const { col.out(p, k * nv + c, v); }
};

template <class T, class Img, class C>
FD void ltdl_solve_vec(const Img& M, const float* LD, const float* b, float* x, const C& col) {
  ltdl_solve_one<T>(M, LD, VecIn<C>{b, col}, VecOut<C>{x, col}, col);
}

// M^-1 column by column (dense, symmetric): nv solves against unit vectors.
template <class T, class Img, class C>
FD void ltdl_inverse(const Img& M, const float* LD, float* Minv, const C& col) {
  const int nv = T::kFree ? T::nb(M) + 5 : T::nb(M);
#pragma unroll 1
  for (int c = 0; c < nv; ++c) ltdl_solve_one<T>(M, LD, UnitIn{c}, ColOut<C>{Minv, c, nv, col}, col);
}

}  // namespace frax
