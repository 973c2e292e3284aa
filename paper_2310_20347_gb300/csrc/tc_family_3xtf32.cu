// Tensor-core family members with mode TC_3XTF32 (see gen_family.py).
#define G3_TU_MODE g3::TC_3XTF32
#define G3_TU_REGISTER register_family_3xtf32
#define G3_TU_REGISTER_GROUPED register_grouped_3xtf32
#include "tc_family_tu.cuh"
