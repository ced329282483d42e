// nh_peel_rs12.cu -- the peel and two-phase kernels instantiated for (r,s) = (1,2).
#include "nh_peel.cuh"

namespace nhp {
NH_PEEL_PAIR(1, 2)
}  // namespace nhp
