// z3_df_p2.cu -- the double-float three-stage Z pass for tiles of 2 row
// classes x 4 columns (z3_df_pass.cuh).
#include "z3_df_pass.cuh"

namespace ctap {

bool launch_z3_df_p2(const ZArgs<df> &a, cudaStream_t st)
{
    return z3df::try_z3<1024, 16, 4, 16, 2, 4>(a, st);
}

}  // namespace ctap
