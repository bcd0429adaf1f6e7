// Internal: device-side generator of the seeded initial field (init_field.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kin {

// splitmix64 output 0 of the stream seeded with `seed` (the field key).
uint64_t field_key(uint64_t seed);

// Unscaled solenoidal Gaussian modes in the half-complex layout [kz][ky][kx],
// kx = 0..N/2, for the three velocity components.
cudaError_t generate_modes(int N, uint64_t seed, double2* u0, double2* u1, double2* u2,
                           cudaStream_t stream);

// u_hat *= shell_scale[shell(n)] * glob for excited modes (0 elsewhere).
cudaError_t scale_modes(int N, const double* shell_scale, double glob, double2* u0, double2* u1,
                        double2* u2, cudaStream_t stream);

}  // namespace kin
