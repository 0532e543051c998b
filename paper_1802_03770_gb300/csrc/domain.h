// The occluded-domain preconditioner (domain.cu): the FD operator on Omega
// with Dirichlet conditions on the hole, applied through the box solve and
// the capacitance matrix of the hole's boundary.
#pragma once

#include "internal.h"

namespace fl {

struct PcgState;

// Largest hole boundary |Gamma| the dense capacitance factor is built for.
constexpr int kMaxGamma = 2048;

// Device data of one capacitance factor.
struct DomainData {
  int m = 0;              // |Gamma|
  int* idx = nullptr;     // linear indices of Gamma in the box (m)
  double* LD = nullptr;   // m x m: L' strictly below the diagonal, D on it
};

// Fills dd.LD with the L D L^T factor of C = E^T B^{-1} E for
// B = shift I + scale C h^d L_box, from m FP64 box solves of unit vectors
// (e and z: N-double scratch; tb's tridiagonal table must hold shift,
// scale).
cudaError_t dom_build_capacitance(const Geo& g, const Tables<double>& tb, const DomainData& dd,
                                  double shift, double scale, double* e, double* z, cudaStream_t s);

// us[Gamma] = -C^{-1} w[Gamma] (FP64 arithmetic); us elsewhere untouched.
// Skipped when st->done (st nullable).
template <typename T>
cudaError_t dom_interface_solve(const DomainData& dd, const T* w, T* us, const PcgState* st,
                                cudaStream_t s);

cudaError_t configure_domain_kernels();

}  // namespace fl
