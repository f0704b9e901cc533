// Outer-path kernel instantiations: batched model shapes (E, C, stochastic C, G, portfolios).
#include "outer.cuh"

namespace cva {

int outer_insts_batched(const OuterInst **out)
{
    static const OuterInst insts[] = {
        {10, 8, 8, 10, 6, outer_launch<10, 8, 8, 10, 6>, outer_forget, nullptr},
    };
    *out = insts;
    return (int)(sizeof(insts) / sizeof(insts[0]));
}

}  // namespace cva
