// Host emulation of the CUDA device built-ins a kernel of the library uses,
// for running kernels on the CPU under AddressSanitizer (tests only): every
// CUDA thread of a block is a std::thread, __syncthreads is a std::barrier,
// the block's dynamic shared memory is a heap buffer of exactly the launch's
// size, and cp.async copies are plain copies.
#pragma once
#define IGAPW_HOST_EMU 1
#include <barrier>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>

struct EmuDim {
    unsigned x = 0, y = 0, z = 0;
};
inline thread_local EmuDim emu_threadIdx, emu_blockIdx, emu_blockDim;
inline thread_local std::barrier<>* emu_barrier = nullptr;
inline thread_local unsigned char* emu_smem_ptr = nullptr;
inline unsigned char* igapw_emu_smem() { return emu_smem_ptr; }
inline void emu_syncthreads() { emu_barrier->arrive_and_wait(); }
template <class T>
inline T emu_ldg(const T* p) { return *p; }
inline int emu_ffs(int x) { return __builtin_ffs(x); }
inline int emu_float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
inline float emu_int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
inline unsigned emu_atomic_or(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_RELAXED); }

#undef __launch_bounds__
#define __launch_bounds__(...)
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline int min(int a, int b) { return a < b ? a : b; }
using std::isfinite;
#define threadIdx emu_threadIdx
#define blockIdx emu_blockIdx
#define blockDim emu_blockDim
#define __syncthreads emu_syncthreads
#define __ldg emu_ldg
#define __ffs emu_ffs
#define __float_as_int emu_float_as_int
#define __int_as_float emu_int_as_float
#define atomicOr emu_atomic_or
