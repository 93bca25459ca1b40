// S-polarised (TMz) instances of the batched blocked kernel: code shapes
// 0-3 and 5 at K = 1..8.
#include "blocked_impl.cuh"

namespace fdtd {

bool launch_blocked_batch_s(const BatchArgs& b, int K, int variant, int step_off, int parity,
                            cudaStream_t st) {
    const unsigned grid = (unsigned)b.n_tasks;
    switch (K) {
#define X(k)                                                                                   \
    case k:                                                                                    \
        if (variant == 3) k_blocked_batch_cap<k, 0><<<grid, 32, 0, st>>>(b, step_off, parity); \
        else if (variant == 2) k_blocked_batch<k, 2, 0><<<grid, 32, 0, st>>>(b, step_off, parity); \
        else if (variant == 5) k_blocked_batch<k, 5, 0><<<grid, 32, 0, st>>>(b, step_off, parity); \
        else if (variant) k_blocked_batch<k, 1, 0><<<grid, 32, 0, st>>>(b, step_off, parity);  \
        else k_blocked_batch<k, 0, 0><<<grid, 32, 0, st>>>(b, step_off, parity);               \
        break;
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return false;
    }
    return true;
}

}  // namespace fdtd
