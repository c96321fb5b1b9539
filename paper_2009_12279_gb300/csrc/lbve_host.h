// lbve_host.h -- host-side helpers shared by the C-ABI translation units.
#pragma once

#include <string>

#include "../../include/lbve.h"
#include "lbve_launch.h"

namespace lbve {
// Relaxation rates and kernel constants of a parameter set (FP64, host arithmetic).
void fill_phys(const lbve_params &p, Phys<double> &ph);
bool params_valid(const lbve_params *p, std::string &why);
int default_block_x(const lbve_params &p);
} // namespace lbve
