// Tensor-core family members with mode TC_F16 (see gen_family.py).
#define G3_TU_MODE g3::TC_F16
#define G3_TU_REGISTER register_family_f16
#define G3_TU_REGISTER_GROUPED register_grouped_f16
#include "tc_family_tu.cuh"
