// nh_peel_rs13.cu -- the peel and two-phase kernels instantiated for (r,s) = (1,3).
#include "nh_peel.cuh"

namespace nhp {
NH_PEEL_PAIR(1, 3)
}  // namespace nhp
