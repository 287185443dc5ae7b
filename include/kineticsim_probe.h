/*
 * kineticsim_probe.h -- roofline probes of the GB300 engine (measurement only).
 *
 * The paper gives no hardware peaks for this method (its kernel is described as
 * arithmetic-bound, Sec. V).  These probes measure the ceilings the persistent
 * kernel is held against: conflict-free shared-memory atomic throughput (one
 * order aggregated per agent-event), 32x32->64-bit product throughput as one
 * wide multiply or as a high-word and a low-word multiply (Philox4x32-10 needs
 * 20 products per agent-event), the Philox block rate of the kernel's own
 * draw routine, the SplitMix64 mix rate of the paper-agent kernel's routine
 * (two mixes per agent-event), and the HBM bandwidth of the kernel's state
 * load and store phases.
 *
 * Conventions as in kineticsim.h: KS_OK on success, work queued on `stream`,
 * the caller times it (CUDA events on the same stream).
 */
#ifndef KINETICSIM_PROBE_H
#define KINETICSIM_PROBE_H

#include <stddef.h>
#include <stdint.h>

#include "kineticsim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ks_probe_kind {
  KS_PROBE_SMEM_RED = 0,  /* red.shared.add.u32, each lane on its own bank; ops = lane-atomics */
  KS_PROBE_MUL_WIDE = 1,  /* independent mad.wide.u32 chains; ops = wide multiplies            */
  KS_PROBE_PHILOX = 2,    /* the kernel's per-agent Philox4x32-10 draw; ops = blocks           */
  KS_PROBE_MUL_HILO = 3,  /* independent chains of 32 x 32 -> 64 products taken as mul.hi and
                             mul.lo (the Philox rounds' form); ops = products                 */
  KS_PROBE_SPLITMIX = 4,  /* the paper-agent kernel's two SplitMix64 mixes per agent-step, in a
                             loop with nothing else; ops = mixes                              */
  KS_PROBE_WAIT_TIMEOUT = 5 /* failure detection, not a roofline: one warpgroup runs the policy
                             path's bounded tensor-core wait on an mbarrier that nothing
                             arrives at (no MMA issued), which must give up after its poll
                             limit (well under a few seconds) and return; `blocks` and
                             `iters` are ignored, uint32 sink[0] receives the error word
                             (0x8 on a timeout) and sink[1] is 1 when the warpgroup stayed
                             aborted for its next wait; ops = 1                             */
} ks_probe_kind;

/* Launches probe `kind` over `blocks` CTAs of 256 threads, `iters` iterations
 * per thread.  `sink` is a device buffer of at least blocks*256*8 bytes that
 * receives values keeping the work observable.  *ops receives the operation
 * count of the launch.  KS_ERR_INVALID_ARG for an unknown kind, zero blocks or
 * NULL pointers. */
ks_status ks_probe(int kind, uint32_t blocks, uint32_t iters, void* sink, void* stream, double* ops);

/* Runs the ensemble's persistent kernel with zero steps: every market's state
 * is loaded into the CTA (orders, inventory, cash, scalars, book rebuild) and
 * stored back unchanged.  *bytes receives the algorithmic state bytes moved
 * (16 B per agent each way plus the per-market scalars). */
ks_status ks_probe_state_io(ks_ensemble* e, void* stream, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* KINETICSIM_PROBE_H */
