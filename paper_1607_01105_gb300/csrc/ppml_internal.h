// Host-side helpers shared by the translation units of libppml.so.
#pragma once
#include <cuda_runtime.h>

#include "../../include/ppml.h"

// Record a formatted message for ppml_last_error() on this thread and return `code`.
int ppml_fail(int code, const char* fmt, ...);
// Clear this thread's message (every public entry point starts with it).
void ppml_clear_error();
// Check cudaGetLastError() after a launch; returns PPML_OK or PPML_E_CUDA.
int ppml_check_launch(const char* what);

// Argument checks shared by the entry points (defined in ppml_grid.cu).
int ppml_validate_desc(const ppml_grid_desc* d);
int ppml_validate_state(const ppml_state* u, const char* what);
// Whether a descriptor has halo faces (a slab of a z-decomposed grid).
int ppml_desc_has_halo(const ppml_grid_desc* d);
// Number of non-NULL low-part pointers of a state (0 or 5 once validated).
int ppml_state_has_lo(const ppml_state* u);

// Isolated-boundary Poisson solver state (ppml_poisson.cu); created on the first solve.
struct PoissonIso;
int ppml_iso_solve(PoissonIso** state, const ppml_grid_desc* d, const void* rho, void* phi,
                   double G, unsigned flags, cudaStream_t st);
void ppml_iso_free(PoissonIso* s);

// Disk Fourier amplitudes (ppml_fourier.cu); buffers created on the first call.
struct FourierState;
int ppml_fourier_run(FourierState** state, const ppml_grid_desc* d, const void* rho, double r_f,
                     int m_max, double* a_out, cudaStream_t st);
void ppml_fourier_free(FourierState* s);
