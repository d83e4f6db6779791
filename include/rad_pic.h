/*
 * rad_pic.h -- C ABI of the small live PIC that drives the diagnostic in situ.
 *
 * Sec. 2.1 sets up the filamentation instability as two equal-density neutral
 * plasma beams streaming through each other in a fully periodic box (units
 * c = m_e = q_e = 1, time in 1/omega_pe); Sec. 2.2 collects the radiation of
 * a subset of the particles while the simulation runs.  This is a compact
 * GPU PIC of that setup so the diagnostic (rad.h) can be driven in situ,
 * step by step, from device-resident particle state:
 *
 *   * 2D3V: an n x n periodic grid of square cells (size d) in the (y, z)
 *     plane, nothing depends on x; particles carry three position and three
 *     momentum components and the box is periodic with L = n d in x, y, z.
 *   * Second-order Yee field solver, dB/dt = -curl E, dE/dt = curl B - J
 *     (eps0 = mu0 = c = 1), with B split in two half steps around the push;
 *     relativistic Boris push with linear (cloud-in-cell) field gather from
 *     the staggered points; charge-conserving current deposition for linear
 *     shapes (Esirkepov), so div E - rho is preserved to rounding.
 *   * FP64 throughout; currents are accumulated with atomics (their order,
 *     and so the last bits of J, varies from run to run).
 *
 * Layouts: fields E, B, J as [3][n][n] (component, y index j, z index k),
 * E_x at node (j, k), E_y at (j+1/2, k), E_z at (j, k+1/2), B_x at
 * (j+1/2, k+1/2), B_y at (j, k+1/2), B_z at (j+1/2, k).  Particles as
 * x, u [3][N] (structure of arrays), species in consecutive ranges.  State
 * after s steps: x_s, u_{s-1/2}, E^s, B^s -- the leapfrog state that call s
 * of rad_accumulate expects.
 *
 * Every call returns RAD_PIC_OK (0) or a negative code; calls are ordered on
 * the stream given at init; pointers may be host or device memory unless
 * stated.  The context owns all its device memory.
 */
#ifndef RAD_PIC_H
#define RAD_PIC_H

#include <stdint.h>

#include "rad.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RAD_PIC_OK 0
#define RAD_PIC_EINVAL (-1)
#define RAD_PIC_ENOMEM (-2)
#define RAD_PIC_ECUDA (-3)
#define RAD_PIC_ERAD (-4) /* the radiation context refused a call (see rad_last_error) */

typedef struct rad_pic rad_pic;

/* A species: count particles (consecutive in x, u), charge q and mass m in
 * units of e and m_e, macro weight w (charge density q w / d^2 per particle). */
typedef struct {
    int64_t count;
    double charge;
    double mass;
    double weight;
} rad_pic_species;

/* n cells per axis (>= 4), cell size d, time step dt (dt < d / 2^(1/2) for
 * the Courant limit, and particles must move less than one cell per step);
 * x, u: [3][N] initial state x_0, u_{-1/2} (N = sum of the counts; positions
 * are wrapped into the box [0, n d)).  Fields start at zero. */
int rad_pic_init(rad_pic **out, int32_t n, double d, double dt, const rad_pic_species *sp,
                 int32_t n_species, const double *x, const double *u, void *cuda_stream);

/* Replace / read E and B ([3][n][n] each; either pointer may be null). */
int rad_pic_set_fields(rad_pic *p, const double *E, const double *B);
int rad_pic_get_fields(rad_pic *p, double *E, double *B);

/* Read the particle state x_s, u_{s-1/2} ([3][N] each; either may be null). */
int rad_pic_get_particles(rad_pic *p, double *x, double *u);

/* Advance n_steps steps. */
int rad_pic_step(rad_pic *p, int32_t n_steps);

/* Steps taken since init. */
int64_t rad_pic_steps_done(const rad_pic *p);

/* Copy particles first .. first + count - 1 of the current state into the
 * device buffers x_out, u_out ([3][count] each): the arguments of one
 * rad_accumulate call. */
int rad_pic_tracked(rad_pic *p, int64_t first, int64_t count, double *x_out, double *u_out);

/* In-situ run: n_steps times, hand the tracked particles (first .. first +
 * count - 1, the radiation context's particles in order; count must equal
 * the context's particle count, else RAD_PIC_EINVAL) to rad_accumulate as
 * call s = rad_pic_steps_done() and advance one step; then hand over the
 * final state too, so every window that ends at the last step closes.  A
 * state the radiation context has already received (the final state of a
 * previous run) is not handed over twice.  Staging buffers are the PIC's. */
int rad_pic_run_coupled(rad_pic *p, rad_ctx *r, int64_t first, int64_t count, int32_t n_steps);

/* Field energy (E^2 + B^2)/2 d^2 summed over the cells and kinetic energy
 * sum w m (gamma - 1), of the current state (host outputs). */
int rad_pic_energy(rad_pic *p, double *field, double *kinetic);

const char *rad_pic_last_error(const rad_pic *p);

void rad_pic_destroy(rad_pic *p);

#ifdef __cplusplus
}
#endif
#endif /* RAD_PIC_H */
