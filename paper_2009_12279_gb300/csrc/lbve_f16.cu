// lbve_f16.cu -- FP16 storage of the shifted, scaled PDFs, FP32 arithmetic.
#include "lbve_table.cuh"

namespace lbve {
const KernelTable *table_f16() { return Launch<__half>::table(2); }
} // namespace lbve
