// Picks the sweep launcher for a plan's precision, tile shape and term count (the
// launchers are compiled separately from sweep_inst.cu, one unit per combination).
#include "kernels.h"

namespace fgt1d {

using SweepFn = cudaError_t (*)(const SweepArgs&, const SweepConsts&, cudaStream_t, cudaEvent_t, int);

#define FGT_SWEEP_SIG (const SweepArgs&, const SweepConsts&, cudaStream_t, cudaEvent_t, int)
#define FGT_DECLARE_SHAPE(p, s)                                                                           \
    cudaError_t sweeps_##p##_s##s##_ne1 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne2 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne3 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne4 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne5 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne6 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne7 FGT_SWEEP_SIG;                                                    \
    cudaError_t sweeps_##p##_s##s##_ne8 FGT_SWEEP_SIG;
#define FGT_ROW(p, s)                                                                                   \
    {sweeps_##p##_s##s##_ne1, sweeps_##p##_s##s##_ne2, sweeps_##p##_s##s##_ne3, sweeps_##p##_s##s##_ne4, \
     sweeps_##p##_s##s##_ne5, sweeps_##p##_s##s##_ne6, sweeps_##p##_s##s##_ne7, sweeps_##p##_s##s##_ne8}

FGT_DECLARE_SHAPE(f64, 0)
FGT_DECLARE_SHAPE(f64, 1)
FGT_DECLARE_SHAPE(f32, 0)
FGT_DECLARE_SHAPE(f32, 1)
FGT_DECLARE_SHAPE(df, 0)
FGT_DECLARE_SHAPE(df, 1)
static_assert(FGT1D_MAX_TERMS == 8, "one launcher per term count 1..8");
static_assert(kNumShapes == 2, "one table row per tile shape");

static const SweepFn kF64[kNumShapes][FGT1D_MAX_TERMS] = {FGT_ROW(f64, 0), FGT_ROW(f64, 1)};
static const SweepFn kF32[kNumShapes][FGT1D_MAX_TERMS] = {FGT_ROW(f32, 0), FGT_ROW(f32, 1)};
static const SweepFn kDF[kNumShapes][FGT1D_MAX_TERMS] = {FGT_ROW(df, 0), FGT_ROW(df, 1)};

static cudaError_t pick(const SweepFn (*table)[FGT1D_MAX_TERMS], const SweepArgs& a, const SweepConsts& c,
                        cudaStream_t st, cudaEvent_t mid, int ev, int shape) {
    if (c.n_e < 1 || c.n_e > FGT1D_MAX_TERMS || shape < 0 || shape >= kNumShapes) return cudaErrorInvalidValue;
    return table[shape][c.n_e - 1](a, c, st, mid, ev);
}

cudaError_t launch_sweeps_f64(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev,
                              int shape) {
    return pick(kF64, a, c, st, mid, ev, shape);
}
cudaError_t launch_sweeps_f32(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int ev,
                              int shape) {
    return pick(kF32, a, c, st, mid, ev, shape);
}
cudaError_t launch_sweeps_df(const SweepArgs& a, const SweepConsts& c, cudaStream_t st, cudaEvent_t mid, int shape) {
    return pick(kDF, a, c, st, mid, 1, shape);
}

}  // namespace fgt1d
