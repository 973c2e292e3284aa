// Tensor-core family members with mode TC_3XBF16 (see gen_family.py).
#define G3_TU_MODE g3::TC_3XBF16
#define G3_TU_REGISTER register_family_3xbf16
#define G3_TU_REGISTER_GROUPED register_grouped_3xbf16
#include "tc_family_tu.cuh"
