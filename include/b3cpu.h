/*
 * b3cpu.h -- C ABI of the host (CPU) engine of the population simulator.
 *
 * What it computes: exactly the step of libb3sim (include/b3sim.h) -- CPG and
 * PD servo, forward kinematics, RNEA bias forces, CRBA mass matrix, Cholesky
 * solve for v_free, box/plane and box/box contacts with the 64-deepest cap,
 * soft projected Gauss-Seidel with disk friction cones, semi-implicit Euler --
 * in FP32 on the host's cores (heights for contact activation in FP64, as on
 * the GPU), one robot at a time per thread, robots handed out to threads from
 * a shared counter.  It shares the model packing, the spatial-algebra helpers
 * and the box/box narrow phase with the GPU kernel (same source), so the two
 * engines take the same geometric decisions.
 *
 * Why it exists: the paper's own contribution (Sec. 6) is a hybrid allocation
 * that runs one part of the variants on the CPU and the rest on the GPU
 * concurrently, in proportion to the measured speed of each.  This library is
 * that CPU side; paper_2502_11129_b300/hybrid.py is the allocator.  It is not
 * a fallback of the GPU simulator: the GPU path never calls it.
 *
 * Conventions are those of b3sim.h: the same sim_config (device, stream,
 * steps_per_launch, warps_per_block and phase_lock are ignored), the same
 * sim_variant_desc, state row strides SIM_QW / SIM_VW / SIM_SW, status bits
 * SIM_ST_*, and status codes SIM_OK / SIM_EINVAL / SIM_ESTATE / SIM_ENOMEM.
 * Every call is synchronous; the caller owns every host buffer.  One context
 * per host thread; cpu_step_n itself runs on `threads` worker threads.
 */
#ifndef B3CPU_H
#define B3CPU_H

#include <stdint.h>

#include "b3sim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpu_ctx cpu_ctx_t;

/* Create a context with a copy of cfg; threads = worker threads for
 * cpu_step_n (0: all hardware threads).  SIM_EINVAL for a bad cfg. */
int cpu_create(const sim_config* cfg, int32_t threads, cpu_ctx_t** out);
int cpu_destroy(cpu_ctx_t* ctx);

/* Replace the population (n >= 1; validated as sim_set_population does, but
 * with at most SIM_WARP_MAX_BODIES bodies per variant: longer chains are
 * stepped by the GPU simulator only).  The state is reset to zero and must be
 * set before stepping. */
int cpu_set_population(cpu_ctx_t* ctx, const sim_variant_desc* v, int32_t n);

/* State rows of variants [first, first + count) (cpg may be NULL: kept);
 * clears their status and records the core xy as the fitness origin. */
int cpu_set_state(cpu_ctx_t* ctx, int32_t first, int32_t count, const float* q, const float* v,
                  const float* cpg);

/* Advance every variant n_steps (>= 0) steps on the worker threads. */
int cpu_step_n(cpu_ctx_t* ctx, int32_t n_steps);

/* State rows and status bits of variants [first, first + count); any output
 * may be NULL. */
int cpu_read_state(cpu_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v, float* cpg,
                   uint32_t* status);

/* Core xy displacement of variants [0, n) since their last cpu_set_state. */
int cpu_fitness(cpu_ctx_t* ctx, float* out, int32_t n);

/* Wall seconds each variant [0, n) (caller's order) took in the last
 * cpu_step_n (0 for a variant that did not step). */
int cpu_robot_seconds(cpu_ctx_t* ctx, double* out, int32_t n);

/* Worker threads of cpu_step_n. */
int cpu_threads(const cpu_ctx_t* ctx);

/* Contacts accumulated over all variants and steps since cpu_set_population. */
int cpu_contacts(cpu_ctx_t* ctx, double* out);

const char* cpu_last_error(const cpu_ctx_t* ctx);

#ifdef __cplusplus
}
#endif
#endif
