/* igs_peaks.h - throughput probes behind the roofline's denominators.
 *
 * libigs_peaks.so measures, on the current CUDA device, the issue rates the
 * rasteriser's roofline is stated against: binary32 fused multiply-add (one
 * per lane, and the packed two-lane form), the special-function unit's
 * exp2 approximation, float and integer min/max, and warp match. It is a
 * measurement aid: the paper has no counterpart and the rasteriser
 * (libimgs.so, imgs.h) does not use it.
 *
 * Every probe launches (SM count x 4) CTAs of 512 threads; each thread runs
 * 8 independent dependency chains of the probed instruction, written as
 * inline PTX. One warm-up launch precedes `reps` timed launches of `iters`
 * x 128 instructions per thread; the fastest launch counts (CUDA events on
 * a private stream). The probe allocates one small device buffer per call.
 */
#ifndef IGS_PEAKS_H
#define IGS_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

enum igs_peak_kind {
  IGS_PEAK_FFMA = 0,   /* fma.rn.f32: one lane-op per thread instruction */
  IGS_PEAK_FFMA2 = 1,  /* fma.rn.f32x2: two lane-ops per thread instruction */
  IGS_PEAK_EX2 = 2,    /* ex2.approx.ftz.f32 on the special-function unit */
  IGS_PEAK_FMNMX = 3,  /* min.f32, two inputs */
  IGS_PEAK_FMNMX3 = 4, /* min.f32, three inputs */
  IGS_PEAK_IMNMX = 5,  /* min.u32 */
  IGS_PEAK_MATCH = 6,  /* match.any.sync.b32 (rate in warp instructions) */
  IGS_PEAK_KINDS = 7
};

/* Runs probe `kind`. On success returns 0 and writes the rate in lane-ops
 * per second (*ops_per_s; packed FFMA counts two per thread instruction),
 * in instructions per second (*instr_per_s; thread instructions, or warp
 * instructions for MATCH) and the fastest launch's time in ms (*best_ms).
 * Returns 1 for an invalid argument, 2 for a CUDA error. */
int igs_peak_probe(int kind, int iters, int reps, double* ops_per_s, double* instr_per_s,
                   float* best_ms);

#ifdef __cplusplus
}
#endif

#endif /* IGS_PEAKS_H */
