// Lattice parameters as the kernels receive them (by value, FP32).
#pragma once

namespace lbm {

// Parameters as the kernels see them (converted from lbm_params on the host).
struct DevParams {
  int nx, ny, pitch, ncomp, nh, periodic_y, powerlaw, mobility, fd_scheme;
  int collapse_h;  // 1: the state holds C_i instead of the populations h^i
  float rho[3], tau[3];
  float pl_n, pl_k, tau_min, tau_max;
  float sig12, sig13, sig23, Lambda, Sig[3], SigT, xi, D0;
  float gravity, force_x;
  long long plane;  // floats per plane (ny * pitch)
};

}  // namespace lbm
