// Tensor-core family members with mode TC_6XBF16 (see gen_family.py).
#define G3_TU_MODE g3::TC_6XBF16
#define G3_TU_REGISTER register_family_6xbf16
#define G3_TU_REGISTER_GROUPED register_grouped_6xbf16
#include "tc_family_tu.cuh"
