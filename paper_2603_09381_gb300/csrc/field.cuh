// Scattered field off the boundaries and its far-field pattern from a
// boundary solution phi = [q_j; u_j] per inclusion (Green's representation
// over all boundaries with the trapezoid rule, G = (i/4) H0(k+ r)).
#pragma once
#include <cuda_runtime.h>
#include "assemble.cuh"

// out[d + c * ndir] = u_inf(angle d) of column c (phi: N x nrhs, ldphi = N).
void far_field(const InclDev* d_inc, NodesDev nodes, int total_nodes, double k0, const double2* phi, int ldphi,
               int nrhs, const double* d_angles, int ndir, double2* out, cudaStream_t st);
// out[p + c * npts] = u^s(xy[2p], xy[2p+1]) of column c.
void scattered_field(const InclDev* d_inc, NodesDev nodes, int total_nodes, double k0, const double2* phi, int ldphi,
                     int nrhs, const double* d_xy, int npts, double2* out, cudaStream_t st);
