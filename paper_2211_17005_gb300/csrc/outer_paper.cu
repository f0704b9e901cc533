// Outer-path kernel instantiations: paper model shapes (E, C, stochastic C, G, portfolios).
#include "outer.cuh"

namespace cva {

int outer_insts_paper(const OuterInst **out)
{
    static const OuterInst insts[] = {
        {10, 8, 8, 10, 1, outer_launch<10, 8, 8, 10, 1>, outer_forget, adjoint_launch<10, 8, 8, 10>},
    };
    *out = insts;
    return (int)(sizeof(insts) / sizeof(insts[0]));
}

}  // namespace cva
