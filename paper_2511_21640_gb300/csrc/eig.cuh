#pragma once
#include "tensor.cuh"

namespace adc {
// Eigen-decomposition of the Hermitian n x n matrix A (overwritten): eigenvalues
// ascending in w[n], eigenvectors in the columns of V (leading dimension ldv).
// info_dev[0] receives the sweep count, or -1 if not converged.
void jacobi_eigh(Exec &ex, cplx *A, int n, int lda, double *w, cplx *V, int ldv, int *info_dev);
// The same decomposition for n <= 128 (eigh_refined_fits): FP32 Jacobi start and
// at least nsteps FP64 refinement steps of the whole decomposition, more until
// the corrections have converged; the FP64 Jacobi when they do not (eig.cu).
// A is not changed.
bool eigh_refined_fits(int n);
void eigh_refined(Exec &ex, const cplx *A, int n, int lda, double *w, cplx *V, int ldv, int nsteps = 3);
// refinement steps of this thread's last eigh_refined call, -1 when it took the FP64 Jacobi
int eigh_refined_last_steps();
}  // namespace adc
