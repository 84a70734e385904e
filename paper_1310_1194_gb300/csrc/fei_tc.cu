// fei_tc.cu -- tensor-core (tcgen05) contraction for p >= 3.  Placeholder
// until the kernel lands: FEI_TC_F16X3 reports FEI_ERR_UNSUPPORTED.
#include "fei_internal.cuh"

namespace fei {

struct TcImage {
  int dummy;
};

fei_status build_tc_image(fei_reference *ref) {
  ref->tc = nullptr;
  return FEI_OK;
}

void free_tc_image(fei_reference *ref) { ref->tc = nullptr; }

fei_status launch_tc_forward(int p, const fei_reference *, const FwdArgs &, int64_t, cudaStream_t) {
  return set_error(FEI_ERR_UNSUPPORTED, "tensor-core path for degree %d not built", p);
}

}  // namespace fei
