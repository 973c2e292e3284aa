// Tensor-core family members with mode TC_I8EMU (see gen_family.py).
#define G3_TU_MODE g3::TC_I8EMU
#define G3_TU_REGISTER register_family_int8emu
#define G3_TU_REGISTER_GROUPED register_grouped_int8emu
#include "tc_family_tu.cuh"
