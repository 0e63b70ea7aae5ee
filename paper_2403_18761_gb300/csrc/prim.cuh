// Device primitives: exclusive scan and LSD radix sort.  All stream-ordered,
// no host synchronisation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Host-side count of kernel launches issued by the library (rpd_launch_count).
void note_launch();

// Exclusive scan: out[i] = sum_{j<i} in[j] for i < n, and out[n] = total.
// tmp must hold scan_tmp_bytes(n).
size_t scan_tmp_bytes(long long n);
void scan_excl(const int32_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s);
void scan_excl(const uint8_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s);
void scan_excl(const int64_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys (at most 64), 8 bits per pass; n < 2^30.  Reads keys_in/vals_in,
// writes keys_out/vals_out.  tmp must hold radix_tmp_bytes(n).  A pass whose
// bounded look-back wait runs out sets *d_err to RPD_E_TIMEOUT (if it is 0).
size_t radix_tmp_bytes(long long n);
void radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                      uint32_t* vals_out, long long n, int bits, void* tmp, int* d_err, cudaStream_t s);
