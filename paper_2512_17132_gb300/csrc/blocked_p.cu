// P-polarised (TEz) instances of the blocked kernel, single runs and
// batches: code shapes 2, 3 and 5 at K = 1..8 (shapes 0 and 1 map to 2).
#include "blocked_impl.cuh"

namespace fdtd {

int blocked_occupancy_p(int K, int variant) {
    switch (K) {
#define X(k)                                                                   \
    case k:                                                                    \
        return variant == 3   ? occupancy_of(k_blocked_cap<k, 1>)                      \
               : variant == 5 ? occupancy_of(k_blocked<k, 5, 1>)                      \
                              : occupancy_of(k_blocked<k, 2, 1>);
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return 0;
    }
}

bool launch_blocked_p(const BlockedArgs& a, int K, int variant, int64_t n0, cudaStream_t st) {
    const unsigned grid = (unsigned)a.n_tasks;
    switch (K) {
#define X(k)                                                                   \
    case k:                                                                    \
        if (variant == 3) k_blocked_cap<k, 1><<<grid, 32, 0, st>>>(a, n0);     \
        else if (variant == 5) k_blocked<k, 5, 1><<<grid, 32, 0, st>>>(a, n0); \
        else k_blocked<k, 2, 1><<<grid, 32, 0, st>>>(a, n0);                   \
        break;
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return false;
    }
    return true;
}

bool launch_blocked_batch_p(const BatchArgs& b, int K, int variant, int step_off, int parity,
                            cudaStream_t st) {
    const unsigned grid = (unsigned)b.n_tasks;
    switch (K) {
#define X(k)                                                                                   \
    case k:                                                                                    \
        if (variant == 3) k_blocked_batch_cap<k, 1><<<grid, 32, 0, st>>>(b, step_off, parity); \
        else if (variant == 5) k_blocked_batch<k, 5, 1><<<grid, 32, 0, st>>>(b, step_off, parity); \
        else k_blocked_batch<k, 2, 1><<<grid, 32, 0, st>>>(b, step_off, parity);               \
        break;
        FDTD_BLOCKED_CASES(X)
#undef X
        default: return false;
    }
    return true;
}

}  // namespace fdtd
