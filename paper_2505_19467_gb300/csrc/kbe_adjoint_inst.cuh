// Explicit instantiations of the reverse mode's per-N_b launchers (internal).
#pragma once

#include "kbe_adjoint_impl.cuh"

// the per-N_b launchers of kbe_adjoint_impl.cuh, instantiated in kbe_adjoint_nb*.cu
#define KBE_ADJ_INSTANCES(PREFIX, NB)                                                                              \
  PREFIX template cudaError_t adj_sweep_nb<NB>(const Mesh &, int, double, const double2 *, const double2 *, const double2 *, double2 *, double2 *, double2 *, double2 *, double2 *, cudaStream_t, int); \
  PREFIX template cudaError_t adj_update_nb<NB>(const Mesh &, int, double, double, const double2 *, const double2 *, const double2 *, const double2 *, const double2 *, const double2 *, const double2 *, double2 *, double2 *, double2 *, double2 *, double2 *, int *, cudaStream_t); \
  PREFIX template cudaError_t adj_products_nb<NB>(bool, const double2 *, const double2 *, double2 *, int, int, double, const double *, const VMat &, double *, cudaStream_t); \
  PREFIX template cudaError_t adj_hvec_nb<NB>(const Mesh &, const HopTable &, const HvecAdj &, const double2 *, cudaStream_t);
