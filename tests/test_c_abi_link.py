"""The library is usable from plain C: a C program that includes include/tf_sals.h and
include/tf_server.h and links libtfsals.so calls the host-only entry points (no GPU
needed)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "tf_sals.h"
#include "tf_server.h"

int main(void) {
    /* Algorithm 3 on 5 rows of one mode over 2 machines */
    const int64_t dims[1] = {5};
    const int64_t nnz0[5] = {7, 1, 4, 4, 2};
    const int64_t *row_nnz[1] = {nnz0};
    int32_t a0[5];
    int32_t *assign[1] = {a0};
    if (tf_assign_rows(TF_SCHED_GREEDY, 1, dims, row_nnz, 2, 0, assign) != TF_OK) return 2;
    /* work items of a mode with one heavy row, 4 bins */
    const int64_t off[4] = {0, 100, 103, 110};
    tf_item items[64];
    int64_t n_items = 0, n_slots = 0, bin_ptr[5];
    if (tf_plan_mode(off, 3, 4, 0, TF_SCHED_LPT, 0, items, 64, &n_items, &n_slots, bin_ptr) != TF_OK)
        return 3;
    int64_t covered = 0;
    for (int64_t i = 0; i < n_items; ++i) covered += items[i].len;
    if (tf_create(NULL, NULL, TF_F32, dims, 0, 0, 1, 0, NULL, 0, NULL) != TF_EINVAL) return 4;
    /* the serving loop's admission decision and the memory estimate, host only */
    const int64_t need[4] = {5, 3, 8, 1};
    int32_t byp[4] = {0, 0, 0, 0}, admit[4];
    const int started = tf_server_plan_admission(4, need, byp, 6, -1, 8, 8, admit);
    const int64_t dims3[3] = {1000, 1000, 100};
    int64_t est = 0;
    if (tf_estimate_bytes(dims3, 3, 100000, 10, 5, TF_F32, 0, 152, &est) != TF_OK) return 5;
    printf("%s|%d %d %d %d %d|%lld %lld %lld|%d %d%d%d%d %d%d%d%d|%lld\n", tf_version(), a0[0],
           a0[1], a0[2], a0[3], a0[4], (long long)n_items, (long long)covered,
           (long long)bin_ptr[4], started, admit[0], admit[1], admit[2], admit[3], byp[0],
           byp[1], byp[2], byp[3], (long long)est);
    return 0;
}
"""


def test_c_program_links_and_calls_host_entry_points():
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    from paper_1410_5209_gb300 import build
    lib = build.build()
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "abi_check.c")
        exe = os.path.join(d, "abi_check")
        with open(src, "w") as f:
            f.write(C_SRC)
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        src, "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.strip()
    version, assign, plan, adm, est = out.split("|")
    assert version.startswith("sals-gb300")
    # rows in the order 0 (7), 2 (4), 3 (4), 4 (2), 1 (1); each to the machine with the
    # fewest entries so far (cap 3 rows): 0 -> m0, 2 -> m1, 3 -> m1, 4 -> m0, 1 -> m1
    assert assign.split() == ["0", "1", "1", "1", "0"]
    n_items, covered, total = map(int, plan.split())
    assert covered == 110 and total == n_items and n_items > 3   # the 100-entry row is split
    # first fit in arrival order with room 6: jobs 0 and 3 start, 1 and 2 are passed once
    assert adm.split() == ["2", "1001", "0110"]
    assert int(est) > 100000 * 4 * 10   # at least values, residual copies, orders, indices
