// Tensor-core family members with mode TC_FP8 (see gen_family.py).
#define G3_TU_MODE g3::TC_FP8
#define G3_TU_REGISTER register_family_fp8
#define G3_TU_REGISTER_GROUPED register_grouped_fp8
#include "tc_family_tu.cuh"
