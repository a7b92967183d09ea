// One translation unit per (B, S) geometry; the build compiles this file once
// per pair with -DSBF_B=<block bits> -DSBF_S=<word bits>, so the kernel
// instantiations are spread over parallel compiler processes.
#include "registry.h"
#include "sbf_register.cuh"

#if !defined(SBF_B) || !defined(SBF_S)
#error "compile with -DSBF_B=<block bits> -DSBF_S=<word bits>"
#endif

#define BLOOMGB_CAT_(a, b, c, d) a##b##c##d
#define BLOOMGB_CAT(a, b, c, d) BLOOMGB_CAT_(a, b, c, d)

namespace bloomgb {
void BLOOMGB_CAT(register_B, SBF_B, _S, SBF_S)(std::vector<KernelEntry>& v) {
  register_geometry<SBF_B, SBF_S>(v);
}
}  // namespace bloomgb
