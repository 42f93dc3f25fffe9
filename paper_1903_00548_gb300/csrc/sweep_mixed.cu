// Mixed-precision block sweep (placeholder until the tensor-core path lands).
#include "sweep_mixed.cuh"

namespace pwqt {

size_t mixed_bytes_per_energy(int, int, int) { return 0; }

int solve_mixed(pwqt_ctx* c, System&, const SweepSys&, std::vector<SweepJob>&, SweepJob*, std::vector<ResJob>&, ResJob*, int,
                int*, cudaStream_t) {
    return fail(c, PWQT_ERR_INVALID_ARG, "mixed precision path not available in this build");
}

}  // namespace pwqt
