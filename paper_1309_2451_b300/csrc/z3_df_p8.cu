// z3_df_p8.cu -- the double-float three-stage Z pass for tiles of 8 row
// classes x 1 column (z3_df_pass.cuh).
#include "z3_df_pass.cuh"

namespace ctap {

bool launch_z3_df_p8(const ZArgs<df> &a, cudaStream_t st)
{
    return z3df::try_z3<1024, 16, 4, 16, 8, 1>(a, st);
}

}  // namespace ctap
