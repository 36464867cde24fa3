// Bounds checks of the checked build (compiled with -DSINDI_CHECKS=1 into
// lib/libsindi_checked.so). Every offset and id a search kernel follows into
// memory is tested first; a failed test sets kErrBounds in the index's error
// word and the access is skipped, so a damaged index or a kernel bug shows up
// as SINDI_ERR_INVALID_DATA on the next check instead of as a fault. Nothing
// traps. In the normal build every test is the constant true and compiles
// away.
//
// The predicates are plain functions of integers so that the host tests can
// run them too.
#pragma once

#include <stdint.h>

#ifndef SINDI_CHECKS
#define SINDI_CHECKS 0
#endif

#ifdef __CUDACC__
#define SINDI_HD __host__ __device__ __forceinline__
#else
#define SINDI_HD inline
#endif

namespace sindi {

constexpr bool kChecks = SINDI_CHECKS != 0;

// A list segment [ps, pe) inside the posting arrays of pcap entries (the
// stored postings rounded up to the 8-entry groups the scan reads).
SINDI_HD bool segment_in_bounds(uint32_t ps, uint32_t pe, uint64_t pcap) { return ps <= pe && pe <= pcap; }

// An 8-aligned group of postings q0 .. q0 + 7 inside the padded arrays.
SINDI_HD bool group_in_bounds(uint32_t q0, uint64_t pcap) { return (q0 & 7u) == 0 && (uint64_t)q0 + 8 <= pcap; }

// A window-local id (shared-memory slot) inside a window of lambda slots.
SINDI_HD bool slot_in_bounds(uint32_t slot, uint32_t lambda) { return slot < lambda; }

// The offsets seg[j * sigma + w] and seg[j * sigma + w + 1] of list I_{j,w}.
SINDI_HD bool list_in_bounds(int32_t j, uint32_t w, int32_t dim, uint32_t sigma) {
    return j >= 0 && j < dim && w < sigma;
}

// A document id (candidate or result) of an index of n documents.
SINDI_HD bool doc_in_bounds(uint32_t id, int64_t n) { return (int64_t)id < n; }

// A document's row [b, e) of the unpruned documents (nnz entries).
SINDI_HD bool row_in_bounds(int64_t b, int64_t e, int64_t nnz) { return 0 <= b && b <= e && e <= nnz; }

}  // namespace sindi
