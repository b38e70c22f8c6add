/*
 * fsm_probe.h -- micro-benchmarks of the GB300 units the surface generator's
 * kernels are bound by (no counterpart in the paper, whose method runs on a
 * CPU; these give the measured denominators of the kernels' rooflines).
 *
 * Each probe runs a kernel that keeps one unit busy -- FP32 fused
 * multiply-add, FP64 fused multiply-add, float<->int conversion, integer
 * ALU, shared-memory loads and shared-memory atomicMin of 32- and 64-bit
 * words with and without bank conflicts -- over every SM, times it with CUDA
 * events and reports the sustained rate. The probes change no device setting
 * (clocks stay as the driver has them): sample the SM clock while they run to
 * state the clock a rate was measured at.
 */
#ifndef FSM_PROBE_H
#define FSM_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Rates of one probe run, in operations per second over the whole GPU
 * (a fused multiply-add counts as 2 flops in the *_flops fields).
 *   fp32_flops        FFMA, 2 flops each
 *   fp64_flops        DFMA, 2 flops each
 *   f2i_ops           float -> int32 conversions (truncating)
 *   i2f_ops           int32 -> float conversions
 *   frnd_ops          float floor (round to integral float)
 *   int_ops           32-bit integer add/xor (independent chains)
 *   lds_ops           32-bit shared-memory loads, conflict-free
 *   atoms32_ops       32-bit shared atomicMin, every lane its own bank
 *   atoms32_conf_ops  32-bit shared atomicMin, 32 lanes on one bank
 *                     (different words: a 32-way bank conflict)
 *   atoms32_same_ops  32-bit shared atomicMin, 32 lanes on one word
 *   atoms64_ops       64-bit shared atomicMin, conflict-free
 *   sms               multiprocessors used
 *   ms_total          device time of all probes */
typedef struct {
    double fp32_flops, fp64_flops;
    double f2i_ops, i2f_ops, frnd_ops, int_ops;
    double lds_ops, atoms32_ops, atoms32_conf_ops, atoms32_same_ops, atoms64_ops;
    int32_t sms, reserved;
    double ms_total;
} fsm_probe_result;

/* Run every probe on `device` (made current for the call; the caller's
 * current device is restored). Returns 0, or a CUDA error code (the out
 * record is then undefined). Each probe is sized to run a few milliseconds;
 * `repeats` >= 1 repetitions of each are timed and the fastest is kept. */
int fsm_probe_run(int device, int repeats, fsm_probe_result* out);

#ifdef __cplusplus
}
#endif
#endif
