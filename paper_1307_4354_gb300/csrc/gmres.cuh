// Restarted GMRES on the device for the coarsest level (gmres.cu).
#pragma once

#include <functional>

#include "ops.cuh"

namespace cpm {

constexpr int kGmresMaxM = 30;  // Krylov dimension per restart (at most)

// Work space of one GMRES solve of n unknowns with Krylov dimension m.
template <typename T>
struct GmresWork {
  int64_t n = 0;
  int m = 0;
  DBuf<T> V, z, zero, r;                 // (m + 1) x n basis, preconditioned vector, 0, residual
  DBuf<double> H, cs, sn, g, y, h, nrm;  // Hessenberg, rotations, rhs, solution, scalars
  DBuf<double> part;                     // block partial dot products
  void alloc(int64_t n, int m);
};

// The level's residual r = f - A u (no partial norms).
template <typename T>
struct GmresOps {
  std::function<void(const T* f, const T* u, T* r, cudaStream_t)> residual;
};

// x = GMRES(m, restarts) solution of A x = b from x = 0, right-preconditioned
// by P = diag(dA) (dA = omega / diag(A)).  Device only, no synchronisation.
template <typename T>
void gmres_solve(const GmresOps<T>& op, GmresWork<T>& G, const T* b, T* x, const T* dA, int restarts,
                 cudaStream_t st);

}  // namespace cpm
