// Packed-key layout build (layout.cu): every coordinate of an entry in one 64-bit key.
#pragma once

#include "common.cuh"

namespace tfs {

// Field of mode m in a packed key: bits [shift[m], shift[m] + bits[m]), bits[m] =
// ceil(log2 I_m); mode 0 is the most significant field.  cnt_off[m] is mode m's first
// slot in the concatenated row-count array.
struct KeyFields {
    int N;
    int shift[kMaxModes];
    int bits[kMaxModes];
    int64_t dims[kMaxModes];
    int64_t cnt_off[kMaxModes];
};

// Sum of the modes' field widths; the packed build applies when it is at most 64.
int packed_key_bits(const int64_t *dims, int N);
KeyFields key_fields(const int64_t *dims, int N);

// Histogram and scan scratch of radix_sort_keys64 (stream-ordered pool allocations).
struct KeySortWorkspace {
    uint32_t *hist = nullptr;
    uint32_t *scan_tmp = nullptr;
    size_t cap_hist = 0, cap_scan = 0;
    void reserve(int64_t n, cudaStream_t st);
    void release(cudaStream_t st);
};
size_t key_sort_workspace_bytes(int64_t n);

// keys[e0 + e] = the packed coordinates of entry e0 + e, e < ne, read from the row-major
// [ne][N] coords of those entries (device); counts[cnt_off[m] + i] += entries with i_m = i
// (counts zeroed by the caller).  A coordinate outside [0, I_m) sets kStatRange and is
// packed and counted as 0.  e0 should be a multiple of pack_count_tile() (not required).
void launch_pack_count(const int32_t *coords, int64_t e0, int64_t ne, const KeyFields &f,
                       uint64_t *keys, uint32_t *counts, DeviceStatus *stat, cudaStream_t st);
int64_t pack_count_tile();

// Stable LSD radix sort of (kin, vin, xin) by key bits [lo_bit, hi_bit) into (kout, vout,
// xout); vin == nullptr stands for 0, 1, ..., n-1; xin is a second payload of xbytes
// (0, 4 or 8) bytes per key, or nothing.  Passes of at most 10 bits alternate between
// the outputs and (kalt, valt, xalt), which must not overlap the input; the input is
// never written.  The alternate buffers go unused when one pass suffices.
void radix_sort_keys64(const uint64_t *kin, const int32_t *vin, const void *xin, uint64_t *kout,
                       int32_t *vout, void *xout, uint64_t *kalt, int32_t *valt, void *xalt,
                       int xbytes, int64_t n, int lo_bit, int hi_bit, KeySortWorkspace &ws,
                       cudaStream_t st);

// What the extraction of one mode writes: for each other mode t (in the layout's
// other-mode order) its field in the key and the degree-rank table that maps the
// field's row id to its slice row, written to oidx[t][j].
struct ExtractArgs {
    int n_other;
    int check_dup;  // 1: flag equal neighbouring keys (kStatDup); the first mode only
    int shift[kMaxModes - 1];
    int bits[kMaxModes - 1];
    int32_t *oidx[kMaxModes - 1];
    const int32_t *rank[kMaxModes - 1];
    // optional: res[j] = x[perm[j]] with xbytes (4 or 8) per value; x == nullptr skips it
    const int32_t *perm;
    const void *x;
    void *res;
    int xbytes;
};

// The other modes' slice rows of every sorted position j < nnz of one mode (and the
// residual copy when a.x is set).
void launch_extract(const uint64_t *keys, int64_t nnz, const ExtractArgs &a, DeviceStatus *stat,
                    cudaStream_t st);

}  // namespace tfs
