/*
 * grpic_oracle.h -- interface of the plain FP64 CPU oracle of the GR PIC step.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this code. It shares no source, header,
 * table or helper with the CUDA library under paper_2511_17701_gb300/.
 *
 * Storage convention (an interface format, kept equal to the CUDA library's so
 * that planes can be compared element by element):
 *   every field plane is a row-major array [NY][NX] of doubles with
 *   NX = n_r + 2*G + 1, NY = n_theta + 2*G + 1, G = 2 ghost cells per side;
 *   grid point (x1, x2) with x1 = i or i+1/2 and x2 = j or j+1/2 is stored at
 *   [j + G][i + G] (a half-integer position is stored at its lower integer).
 */
#ifndef GRPIC_ORACLE_H
#define GRPIC_ORACLE_H
#include <stdint.h>

#define ORA_G 2

enum {
  ORA_B1, ORA_B2, ORA_B3, ORA_D1, ORA_D2, ORA_D3,       /* em   : B^{n-1/2}, D^n      */
  ORA_B01, ORA_B02, ORA_B03, ORA_D01, ORA_D02, ORA_D03, /* em0  : B^{n-3/2}, D^{n-1}  */
  ORA_J1, ORA_J2, ORA_J3,                               /* cur  : J^{n+1/2}           */
  ORA_J01, ORA_J02, ORA_J03,                            /* cur0 : J^{n-1/2}           */
  ORA_BN1, ORA_BN2, ORA_BN3,                            /* B^n (predict output)       */
  ORA_BI1, ORA_BI2, ORA_BI3, ORA_DI1, ORA_DI2, ORA_DI3, /* initial field (MATCH target) */
  ORA_JA1, ORA_JA2, ORA_JA3,                            /* sum of |deposit terms|     */
  ORA_NPLANES
};

typedef struct {
  int metric;          /* 0: flat spacetime (kerr_schild_0), 1: Kerr-Schild           */
  double a;            /* spin (ignored for metric 0)                                  */
  int n_r, n_th;       /* cells in x1 (radial) and x2 (polar)                          */
  double r_min, r_max; /* radial extent; x1 -> r = r0 + (r_min - r0) exp(x1 dxi)      */
  double dt;           /* time step                                                    */
  int n_iter;          /* fixed iteration count of both implicit pushes                */
  double small_angle;  /* SMALL_ANGLE_GR                                               */
  int n_f;             /* number of current filters (sets the horizon layer)           */
  double r_absorb;     /* start of the absorbing (MATCH) layer                         */
  double absorb_coef;  /* strength of the absorbing layer                              */
  double r0, h0;       /* quasi-spherical map (App. A): r = r0 + exp(xi), theta(eta) with
                          the equatorial concentration h0; 0, 0 = plain log-r, uniform theta */
} ora_params;

typedef struct {
  double r, th;                      /* physical coordinates used (theta maybe clamped)  */
  double f, g;                       /* dr/dx1, dtheta/dx2                                */
  double h11, h22, h33, h13;         /* covariant spatial metric, code units              */
  double H11, H22, H33, H13;         /* contravariant spatial metric, code units          */
  double alpha, beta1, sqrt_h, sqrt_ht;
  double d1H11, d1H22, d1H33, d1H13, d1alpha, d1beta1;
  double d2H11, d2H22, d2H33, d2H13, d2alpha, d2beta1;
} ora_metric;

typedef struct {
  int64_t n;
  int32_t *i1, *i2;
  double *dx1, *dx2, *u1, *u2, *u3, *phi, *w;
  uint8_t *tag;                      /* 1 alive, 2 left the domain this step, 0 dead      */
  int32_t *i1p, *i2p;
  double *dx1p, *dx2p;
  double qm;                         /* Lorentz coefficient (q/m) per unit stored field   */
  double qc;                         /* deposit coefficient (sign of q included)          */
  int massless;                      /* 1: massless (Sec. 2.3: gamma = sqrt(h^ij u_i u_j), no
                                        EM push, Sec. 3.1); neutral, so nothing deposited  */
} ora_species;

#endif
