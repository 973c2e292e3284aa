// Tensor-core family members with mode TC_BF16 (see gen_family.py).
#define G3_TU_MODE g3::TC_BF16
#define G3_TU_REGISTER register_family_bf16
#define G3_TU_REGISTER_GROUPED register_grouped_bf16
#include "tc_family_tu.cuh"
