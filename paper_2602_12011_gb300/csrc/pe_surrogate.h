// pe_surrogate.h -- types shared by the surrogate kernels and host code (pe_surrogate.cu).
#pragma once

namespace pe {

// Training box of the surrogate: samples inside it take the surrogate path, the rest the plain
// generator (fallback).
struct SurBox {
  double mlo, mhi;   // total mass range [Msun]
  double qmax;       // largest mass ratio
  double chimax;     // largest |chi_i|
  double qnet;       // largest mass ratio whose node values come from the network (exact above)
};

}  // namespace pe
