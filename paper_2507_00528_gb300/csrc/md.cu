// Molecular dynamics with the model's forces (forward-only inference):
// velocity-Verlet updates of positions and velocities, and wrapping of the
// positions back into their periodic cell.  Units: A, fs, amu, eV.
#include "gnep_internal.h"

namespace gnep {

namespace {

// 1 eV / (A amu) in A / fs^2: the electronvolt (1.602176634e-19 J) over 1e-10 m
// times the atomic mass unit (1.66053906660e-27 kg), in m / s^2, times 1e-20.
constexpr double kAccel = 1.602176634e-19 / (1e-10 * 1.66053906660e-27) * 1e-20;

// Inverse cell per structure (rows a, b, c of H are the lattice vectors).
__global__ void k_md_hinv(int S, const double* __restrict__ cell, double* __restrict__ hinv) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double* H = cell + 9 * s;
  const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                     H[2] * (H[3] * H[7] - H[4] * H[6]);
  const double id = 1.0 / det;
  double* o = hinv + 9 * s;
  o[0] = (H[4] * H[8] - H[5] * H[7]) * id;
  o[1] = (H[2] * H[7] - H[1] * H[8]) * id;
  o[2] = (H[1] * H[5] - H[2] * H[4]) * id;
  o[3] = (H[5] * H[6] - H[3] * H[8]) * id;
  o[4] = (H[0] * H[8] - H[2] * H[6]) * id;
  o[5] = (H[2] * H[3] - H[0] * H[5]) * id;
  o[6] = (H[3] * H[7] - H[4] * H[6]) * id;
  o[7] = (H[1] * H[6] - H[0] * H[7]) * id;
  o[8] = (H[0] * H[4] - H[1] * H[3]) * id;
}

// v += dt/2 F/m, x += dt v, then x is wrapped into the cell: f = x H^-1,
// f -= floor(f), x = f H.
__global__ void k_md_kick_drift(int N, const int* __restrict__ atom_struct, const double* __restrict__ cell,
                                const double* __restrict__ hinv, double* __restrict__ pos, double* __restrict__ vel,
                                const double* __restrict__ inv_mass, const float* __restrict__ F, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int s = atom_struct[i];
  const double a = 0.5 * dt * kAccel * inv_mass[i];
  double x[3];
  for (int c = 0; c < 3; ++c) {
    const double v = vel[3 * (size_t)i + c] + a * (double)F[3 * (size_t)i + c];
    vel[3 * (size_t)i + c] = v;
    x[c] = pos[3 * (size_t)i + c] + dt * v;
  }
  const double* inv = hinv + 9 * s;
  const double* H = cell + 9 * s;
  double f[3];
  for (int c = 0; c < 3; ++c) {
    f[c] = x[0] * inv[c] + x[1] * inv[3 + c] + x[2] * inv[6 + c];
    f[c] -= floor(f[c]);
  }
  for (int c = 0; c < 3; ++c) pos[3 * (size_t)i + c] = f[0] * H[c] + f[1] * H[3 + c] + f[2] * H[6 + c];
}

// v += dt/2 F/m
__global__ void k_md_kick(int N, double* __restrict__ vel, const double* __restrict__ inv_mass,
                          const float* __restrict__ F, double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = 0.5 * dt * kAccel * inv_mass[i];
  for (int c = 0; c < 3; ++c) vel[3 * (size_t)i + c] += a * (double)F[3 * (size_t)i + c];
}

}  // namespace

int md_kick_drift(const gnep_nlist* nl, double* pos, double* vel, const double* inv_mass, const float* F, double dt,
                  cudaStream_t st) {
  const int N = nl->n_atoms, S = nl->n_struct;
  if (N == 0) return GNEP_OK;
  double* hinv = nullptr;
  GNEP_CUDA(cudaMallocAsync(&hinv, sizeof(double) * 9 * (size_t)S, st));
  k_md_hinv<<<blocks_for(S, 128), 128, 0, st>>>(S, nl->cell, hinv);
  k_md_kick_drift<<<blocks_for(N, 256), 256, 0, st>>>(N, nl->atom_struct, nl->cell, hinv, pos, vel, inv_mass, F, dt);
  GNEP_CHECK_LAUNCH("k_md_kick_drift");
  GNEP_CUDA(cudaFreeAsync(hinv, st));
  return GNEP_OK;
}

int md_kick(const gnep_nlist* nl, double* vel, const double* inv_mass, const float* F, double dt, cudaStream_t st) {
  const int N = nl->n_atoms;
  if (N == 0) return GNEP_OK;
  k_md_kick<<<blocks_for(N, 256), 256, 0, st>>>(N, vel, inv_mass, F, dt);
  GNEP_CHECK_LAUNCH("k_md_kick");
  return GNEP_OK;
}

}  // namespace gnep
