// Helpers shared by the LJ pair kernels (forces.cu, lj_tile.cu).
#pragma once

namespace r3b {

// Cell offset of a pair-list entry: (c - 1) for the 2-bit code c of one axis (0, 1, 2; 3 in padding
// entries), exactly, from the bits of an FP32 number (2^23 + c minus 2^23 + 1): no table lookup.  The
// offset times the cell edge is exact, so (pj - pi) + offset rounds once, as with a table of offsets.
#ifndef R3B_LJ_ARITH_OFF
#define R3B_LJ_ARITH_OFF 1
#endif
__device__ __forceinline__ float off_unit(unsigned c) { return __int_as_float(0x4B000000u | c) - 8388609.0f; }

}  // namespace r3b
