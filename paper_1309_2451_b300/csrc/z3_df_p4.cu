// z3_df_p4.cu -- the double-float three-stage Z pass for tiles of 4 row
// classes x 2 columns (z3_df_pass.cuh).
#include "z3_df_pass.cuh"

namespace ctap {

bool launch_z3_df_p4(const ZArgs<df> &a, cudaStream_t st)
{
    return z3df::try_z3<1024, 16, 4, 16, 4, 2>(a, st);
}

}  // namespace ctap
