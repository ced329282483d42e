// nh_peel_rs34.cu -- the peel and two-phase kernels instantiated for (r,s) = (3,4).
#include "nh_peel.cuh"

namespace nhp {
NH_PEEL_PAIR(3, 4)
}  // namespace nhp
