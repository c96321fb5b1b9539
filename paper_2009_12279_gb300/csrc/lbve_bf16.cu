// lbve_bf16.cu -- BF16 storage of the shifted PDFs, FP32 arithmetic.
#include "lbve_table.cuh"

namespace lbve {
const KernelTable *table_bf16() { return Launch<__nv_bfloat16>::table(3); }
} // namespace lbve
