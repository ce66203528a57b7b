// Inner-tolerance policy of the mixed-precision refinement, shared by
// pb_solve (solve.cu) and the request server (serve.cu). Plain C++ (no CUDA):
// the host tests compile it on its own.
#pragma once

#include <algorithm>

namespace pb {

// Mixed-precision refinement: an inner solve asks for
// min(INNER_CAP, max(inner_tol, INNER_AIM x tol / rel)) relative to the
// current outer residual rel. The FP32 operator's own error on the rough
// corrections of later sweeps (the treecode's and FP32 rounding's) caps every
// sweep's reduction at a few per cent, so an inner solve that asks for much
// more than the tolerance needs only spends iterations: with an aim of 1 and a
// cap of 0.1 the three workloads measured (the 20-charge sphere, the 500- and
// 5,000-atom molecules) take 1 to 3 fewer iterations than with an aim of 0.2
// and a cap of 0.5, in the same number of sweeps; an aim of 2 or more let the
// last sweep land above the tolerance on the 500-atom molecule (one sweep more).
constexpr double INNER_AIM = 1.0;
constexpr double INNER_CAP = 0.1;
constexpr double INNER_RETRY = 1e-3;

// Inner tolerance of the next refinement sweep after `sweeps` sweeps whose
// outer residuals were prev and then rel, the last sweep having asked its
// inner solve for inner_last; negative when the refinement should stop
// because the outer residual no longer falls (less than a halving) although
// the last inner solve asked for a reduction of INNER_RETRY or better (the
// residual's own accuracy is reached). A sweep that stalled on a looser inner
// solve (a Calderon preconditioner's FP32 operator, say, can make a sweep
// contract by less than the inner solve did) is followed by one that asks for
// INNER_RETRY.
inline double refine_inner_tol(int sweeps, double rel, double prev, double inner_last, double tol,
                               double inner_min) {
    const double inner = std::min(INNER_CAP, std::max(inner_min, INNER_AIM * tol / rel));
    if (sweeps < 2 || rel <= 0.5 * prev) return inner;
    if (inner_last <= std::max(INNER_RETRY, inner_min)) return -1.0;
    return std::max(inner_min, std::min(inner, INNER_RETRY));
}

}  // namespace pb
