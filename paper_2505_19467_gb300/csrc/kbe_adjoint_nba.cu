// Reverse-mode launchers for N_b in {1, 2, 3, 4} (see kbe_adjoint_impl.cuh); the
// reverse mode is split by N_b over several translation units so that they
// compile in parallel.
#include "kbe_adjoint_inst.cuh"

namespace kbe {

KBE_ADJ_INSTANCES(, 1)
KBE_ADJ_INSTANCES(, 2)
KBE_ADJ_INSTANCES(, 3)
KBE_ADJ_INSTANCES(, 4)

}  // namespace kbe
