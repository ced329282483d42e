// nh_peel_rs24.cu -- the peel and two-phase kernels instantiated for (r,s) = (2,4).
#include "nh_peel.cuh"

namespace nhp {
NH_PEEL_PAIR(2, 4)
}  // namespace nhp
