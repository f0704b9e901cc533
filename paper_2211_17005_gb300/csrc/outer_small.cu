// Outer-path kernel instantiations: small model shapes (E, C, stochastic C, G, portfolios).
#include "outer.cuh"

namespace cva {

int outer_insts_small(const OuterInst **out)
{
    static const OuterInst insts[] = {
        {1, 2, 0, 5, 1, outer_launch<1, 2, 0, 5, 1>, outer_forget, adjoint_launch<1, 2, 0, 5>},
        {1, 2, 0, 10, 1, outer_launch<1, 2, 0, 10, 1>, outer_forget, adjoint_launch<1, 2, 0, 10>},
    };
    *out = insts;
    return (int)(sizeof(insts) / sizeof(insts[0]));
}

}  // namespace cva
