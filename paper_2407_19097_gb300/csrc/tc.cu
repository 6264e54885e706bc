// Tensor-core (tcgen05) convolutions -- placeholder until the kernels land.
#include "net.h"

namespace nrv {

nrv_status tc_repack(Net*, cudaStream_t) { return NRV_OK; }

nrv_status tc_conv3(const Net*, int, const void*, int, const void*, int, void*, const Geo&, int,
                    nrv_prec, cudaStream_t) {
    return fail(NRV_ERR_UNSUPPORTED, "no tensor-core kernel for this shape");
}

}  // namespace nrv
