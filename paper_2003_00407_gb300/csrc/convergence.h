// Stopping test of one CheFSI pass for one element (Alg. CheFSI: the loop runs until the residuals of
// the wanted Ritz pairs meet the tolerance).  Shared by the device bookkeeping kernel and the host
// entry point dgdft_stage_converged, so both apply the same rule.
//
// FP64 stage: leave when the largest residual of the first n_eig Ritz pairs is <= tol (or not finite).
// FP32 stage of the mixed path: also leave when it is <= tol_mixed, or when it has stagnated -- two
// consecutive passes that each reduce it by less than 20% and end at a level that FP32 rounding explains:
//     max_resid <= kFp32FloorFactor * 2^-24 * |b_up|
// (b_up bounds the spectrum of H, so 2^-24 |b_up| is the rounding level of an FP32 application of H; on
// the 32x32x48 sheet elements the stagnation level is about 3 times that).  Stagnation above that level
// is slow convergence, not the FP32 floor: the element keeps iterating, up to max_iter.
#pragma once

namespace dgdft {

constexpr double kFp32FloorFactor = 32.0;
constexpr double kFp32Eps = 5.9604644775390625e-08;   // 2^-24

// Updates prev_res / stall and returns 1 when the element leaves the stage.
__host__ __device__ inline int stage_converged(double mx, double tol, double tol_mixed, int mixed, double b_up,
                                               double* prev_res, int* stall) {
  const bool finite = mx == mx && mx < 1.0e300;
  int done = (!finite || mx <= tol) ? 1 : 0;
  if (mixed) {
    if (mx <= tol_mixed) done = 1;
    const double floor_level = kFp32FloorFactor * kFp32Eps * (b_up < 0 ? -b_up : b_up);
    if (mx > 0.8 * *prev_res && mx <= floor_level) *stall += 1;   // a stalled pass at the floor level
    else *stall = 0;
    if (*stall >= 2) done = 1;
  }
  *prev_res = mx;
  return done;
}

}  // namespace dgdft
