// bn_sums.cu -- launch geometry of the 2-D fused operator kernels (bn_fused2d*.cu): how many
// CTAs (rows of per-CTA partial sums) one evaluation uses.  The 3-D and CIRCULAR operator has its
// own plan (bn_opnd.cu).
#include <algorithm>

#include "bn_internal.cuh"

namespace bn {

int triple_partials(const bn_solver* s) {
    // opt in to large dynamic shared memory once, outside any stream capture
    configure_fused2d();
    int dev = s->device, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    // resident CTAs per SM of the fused kernel, limited by its shared memory (227 KB per SM usable)
    const size_t smem = fused2d_smem(s->g.N, s->opt.precision);
    const int per_sm = std::max(1, std::min(4, (int)((227 * 1024) / (smem + 1024))));
    return std::max(1, std::min(s->work.count, per_sm * sms));
}

}  // namespace bn
