// lbve_f32.cu -- FP32 storage and arithmetic.  The FP16 and BF16 storage modes (also with
// FP32 arithmetic) have units of their own, so that the three compile in parallel.
#include "lbve_table.cuh"

namespace lbve {
const KernelTable *table_f32() { return Launch<float>::table(1); }
} // namespace lbve
