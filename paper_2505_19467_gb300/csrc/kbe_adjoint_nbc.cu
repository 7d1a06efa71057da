// Reverse-mode launchers for N_b = 12 (see kbe_adjoint_impl.cuh); the
// reverse mode is split by N_b over several translation units so that they
// compile in parallel.
#include "kbe_adjoint_inst.cuh"

namespace kbe {

KBE_ADJ_INSTANCES(, 12)

}  // namespace kbe
