// a1 (split precision): leaf Grams on tcgen05 tensor cores, BF16 hi/lo
// split with three products and FP32 accumulation in TMEM.
#include "common.cuh"
#include "internal.h"

namespace krp {

bool launch_tree_leaves_tc(krp_sampler* s, int j, int LB, int G, int64_t ctas, float* top, size_t smem_fp32) {
    (void)s; (void)j; (void)LB; (void)G; (void)ctas; (void)top; (void)smem_fp32;
    return false;
}

}  // namespace krp
