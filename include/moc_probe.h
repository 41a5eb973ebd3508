/*
 * moc_probe.h -- hardware rate probes of the GB300 MOC library: the denominators its sweeps are
 * measured against.
 *
 * The paper has no counterpart. The planar flat-source sweep (Eq. MOC_sol over every track,
 * polar angle and group, Sec. 3.1) is bound by FP32 arithmetic and by the L2 atomic units that
 * receive its region tallies, not by HBM bandwidth; these probes measure those two rates on the
 * device the library runs on, so that a sweep's roofline fraction can be stated against a
 * measured rate beside the rate derived from unit counts and clocks.
 *
 * Conventions: as in moc_gb300.h (status codes MOC_OK / MOC_ERR_ARG / MOC_ERR_CUDA / MOC_ERR_OOM,
 * no exceptions across the ABI). Every probe is a fixed, bounded amount of work (no waits, no
 * spin loops) on its own stream; the call is synchronous and allocates its scratch buffer with
 * cudaMalloc for the duration of the call only.
 */
#ifndef MOC_PROBE_H
#define MOC_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Probe kinds. "Lane operation" = one thread's instance of the instruction.
 *  MOC_PROBE_FFMA        FP32 fused multiply-adds per second (8 independent chains per thread)
 *  MOC_PROBE_DFMA        FP64 fused multiply-adds per second
 *  MOC_PROBE_RED_F32     red.add.f32 (result unused), every lane in its own 32-byte sector
 *  MOC_PROBE_RED_F32X2   red.add.v2.f32 (8 bytes), every lane in its own sector
 *  MOC_PROBE_RED_F32X4   red.add.v4.f32 (16 bytes), every lane in its own sector
 *  MOC_PROBE_RED_F32X4_PAIR  red.add.v4.f32, lanes 2j and 2j+1 fill one 32-byte sector
 *  MOC_PROBE_RED_F32_ROW8    red.add.f32, 8 consecutive lanes fill one 32-byte sector
 *  MOC_PROBE_ATOM_F32    atom.add.f32 whose old value is consumed (the compensated tally's form)
 *  MOC_PROBE_RED_F64     red.add.f64, every lane in its own sector
 *  MOC_PROBE_RED_F32X4_HBM   as RED_F32X4 over a buffer much larger than L2 (4 GiB)
 *  The atomic probes target a 64 MiB buffer (it stays in L2) except the last, at pseudo-random
 *  sectors (a hash of thread and iteration). */
enum {
  MOC_PROBE_FFMA = 0,
  MOC_PROBE_DFMA = 1,
  MOC_PROBE_RED_F32 = 2,
  MOC_PROBE_RED_F32X2 = 3,
  MOC_PROBE_RED_F32X4 = 4,
  MOC_PROBE_RED_F32X4_PAIR = 5,
  MOC_PROBE_RED_F32_ROW8 = 6,
  MOC_PROBE_ATOM_F32 = 7,
  MOC_PROBE_RED_F64 = 8,
  MOC_PROBE_RED_F32X4_HBM = 9,
  MOC_PROBE_COUNT = 10
};

/* Run probe `kind` on `device`: lane_ops_per_s = lane operations per second (best of 3 timed
 * launches after one warm-up, CUDA events on the probe's stream); sectors_per_s = 32-byte L2
 * sectors touched per second (atomic probes; 0 for the FMA probes); sm_count = the device's
 * multiprocessor count. Any output pointer may be NULL. Errors: MOC_ERR_ARG (unknown kind or
 * device), MOC_ERR_OOM, MOC_ERR_CUDA. */
int moc_probe_rate(int device, int kind, double *lane_ops_per_s, double *sectors_per_s, int *sm_count);

#ifdef __cplusplus
}
#endif

#endif /* MOC_PROBE_H */
