// lbve_f64.cu -- FP64 storage and arithmetic (parity mode).  Built with FMA contraction
// off so that every expression rounds exactly as it is written.
#include "lbve_table.cuh"

namespace lbve {
const KernelTable *table_f64() { return Launch<double>::table(0); }
} // namespace lbve
