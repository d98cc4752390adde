// Lattice parameters as the kernels receive them (by value, FP32).
#pragma once

namespace lbm {

// Parameters as the kernels see them (converted from lbm_params on the host).
struct DevParams {
  int nx, ny, pitch, ncomp, nh, periodic_y, powerlaw, mobility, fd_scheme;
  int collapse_h;  // 1: the state holds C_i instead of the populations h^i
  int g16;         // 1: g stored as FP16 deviations (with collapse_h)
  int open_x;      // 1: velocity inlet at x = 0, convective outlet at x = nx - 1
  float u_in, c_in[2];
  float g16_scale, g16_inv_scale;
  float rho[3], tau[3];
  float pl_n, pl_k, tau_min, tau_max;
  float sig12, sig13, sig23, Lambda, Sig[3], SigT, xi, D0;
  float gravity, force_x;
  // precomputed on the host (double, then rounded)
  float inv_sig[3];    // 1 / Sigma_i
  float mu_pre;        // 4 Sigma_T / xi (Eq. 5)
  float grad_coef[3];  // (3/4) xi Sigma_i (Eq. 5)
  float d0_sig[3];     // D0 / Sigma_i (Eq. 6)
  float n1, k3;        // n - 1 and k / cs^2 (Eq. 31-32)
  float n1h;           // (n - 1) / 2
  long long plane;  // floats per plane (ny * pitch)
};

}  // namespace lbm
