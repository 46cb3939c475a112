// Host build of the 3D element physics of the CUDA library (the same header the
// kernels compile), so tests can compare it with the FP64 oracle on the CPU.
#include "../../paper_1907_01252_gb300/csrc/fsi_element3d.cuh"

extern "C" int fsi3_cell_residual_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                       int solid, int outflow, double k, double theta, double alpha, double* Re) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  fsi3::cell_residual3(P, T, Ue, Uo, h, solid != 0, outflow != 0, k, theta, alpha, Re);
  return 0;
}

extern "C" int fsi3_cell_jacobian_host(const double* phys, const double* Ue, const double* Uo, const double* h,
                                       int solid, int outflow, double k, double theta, double alpha, double* Ke) {
  static fsi3::Tables3 T;
  static bool ready = false;
  if (!ready) {
    fsi3::build_tables3(T);
    ready = true;
  }
  const fsi3::Phys3 P{phys[0], phys[1], phys[2], phys[3], phys[4]};
  fsi3::cell_jacobian3(P, T, Ue, Uo, h, solid != 0, outflow != 0, k, theta, alpha, Ke);
  return 0;
}
