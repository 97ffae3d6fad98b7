// Interface of the Rayleigh-Ritz solver shared by the LOBPCG driver: three kernels (a
// one-CTA reduction to tridiagonal form, one warp per eigenpair, a one-CTA finish) that
// hand their intermediate results over in a device scratch area.
#pragma once
#include <cuda_runtime.h>

#define RR_MMAX 96
#define RR_KMAX 32
#define RR_LD 97            // padded leading dimension of the m x m work matrices
#define RR_LDF 97           // leading dimension of the FP32 m x m matrices

// Hand-over between the kernels of one Rayleigh-Ritz solve (device memory).
struct RRScratch {
  double MA[RR_MMAX * RR_LD];        // M (lower triangle) and R^T (strict upper)
  float J[RR_MMAX * RR_LDF];         // Householder vectors below the subdiagonal
  float V[RR_MMAX * RR_LDF];         // FP32 eigenvectors of M (columns)
  double sc[RR_MMAX], rdg[RR_MMAX];  // unit-diagonal scaling, 1 / diag(R)
  float dd[RR_MMAX], ee[RR_MMAX], e2[RR_MMAX], bet[RR_MMAX], lam[RR_MMAX];
  float lo, hi, tn;                  // Gershgorin interval of T, max |bound|
  int m, dropped;                    // order used (P dropped: m_nop), whether P was dropped
};

// G: [2][m][m] (G_A then G_B, row stride m).  Outputs: C [m][k] (coefficients of the k
// lowest Ritz vectors in the basis of G, rows past m_nop are 0 when P was dropped),
// theta [k] ascending, optional theta_hist [k] copy, optional Cp [m][k] (coefficients
// of the next P, B-orthogonal to the Ritz vectors).  *status must be 0 on entry
// (nonzero: the kernel does nothing); it becomes 2 for a dependent basis that dropping P
// does not cure and 3 for a non-finite Ritz value.  *restarts (optional) counts drops.
struct RRParams {
  const double* G;
  int m, k, m_nop;
  double* C;
  double* Cp;
  double* theta;
  double* theta_hist;
  int* status;
  int* restarts;
  RRScratch* scr;      // device scratch of one solve (reused in stream order)
};

int bf_rr_launch(const RRParams& a, cudaStream_t s);
