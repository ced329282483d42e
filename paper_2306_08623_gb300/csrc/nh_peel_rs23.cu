// nh_peel_rs23.cu -- the peel and two-phase kernels instantiated for (r,s) = (2,3).
#include "nh_peel.cuh"

namespace nhp {
NH_PEEL_PAIR(2, 3)
}  // namespace nhp
