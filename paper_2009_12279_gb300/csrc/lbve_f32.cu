// lbve_f32.cu -- FP32 arithmetic with FP32, FP16 or BF16 storage of the shifted PDFs.
#include "lbve_table.cuh"

namespace lbve {
const KernelTable *table_f32() { return Launch<float>::table(1); }
const KernelTable *table_f16() { return Launch<__half>::table(2); }
const KernelTable *table_bf16() { return Launch<__nv_bfloat16>::table(3); }
} // namespace lbve
