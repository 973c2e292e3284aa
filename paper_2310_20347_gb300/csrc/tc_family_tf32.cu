// Tensor-core family members with mode TC_TF32 (see gen_family.py).
#define G3_TU_MODE g3::TC_TF32
#define G3_TU_REGISTER register_family_tf32
#define G3_TU_REGISTER_GROUPED register_grouped_tf32
#include "tc_family_tu.cuh"
