"""The public header as plain C: a C99 program includes include/fsz.h, links against the
library and calls its host-only entry points (no GPU needed: none of them makes a CUDA
call). The struct layouts it sees must be the ones the Python binding declares."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "fsz.h"

int main(void) {
  unsigned char bad[64];
  fsz_schedule sc;
  uint64_t n = 0;
  memset(bad, 0, sizeof(bad));
  printf("sizes %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fsz_dims), sizeof(fsz_cfield),
         sizeof(fsz_dfield), sizeof(fsz_schedule), sizeof(fsz_quality), sizeof(fsz_server_config),
         sizeof(fsz_request), sizeof(fsz_completion), sizeof(fsz_server_stats));
  printf("offsets %zu %zu %zu\n", offsetof(fsz_cfield, eb), offsetof(fsz_cfield, out_bytes),
         offsetof(fsz_dfield, out_capacity_elems));
  printf("version %s\n", fsz_version());
  printf("bound %llu %llu\n", (unsigned long long)fsz_compress_bound(1000),
         (unsigned long long)fsz_compress_bound(0));
  printf("workspace %llu\n", (unsigned long long)fsz_workspace_bytes(1u << 20));
  printf("header %d\n", (int)fsz_read_header(bad, &n, NULL, NULL, NULL, NULL));
  if (fsz_set_schedule_ex(NULL) != FSZ_OK || fsz_get_schedule(&sc) != FSZ_OK) return 2;
  printf("schedule %u %u %u %u %u %u %u %u\n", sc.stats_ctas_per_sm, sc.compress_ctas_per_sm,
         sc.decompress_ctas_per_sm, sc.compress_ticket_chunks, sc.compress_ticket_lead,
         sc.decompress_ticket_chunks, sc.decompress_records, sc.min_tickets_per_cta);
  sc.decompress_records = 1; /* below twice the ticket: refused, schedule unchanged */
  printf("refused %d\n", (int)fsz_set_schedule_ex(&sc));
  return 0;
}
"""


def test_header_compiles_as_c_and_links(fszlib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_fsz.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_fsz"
    libdir = os.path.dirname(fszlib.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(fszlib.LIB_PATH),
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    lines = dict(line.split(" ", 1) for line in out.strip().splitlines())

    from paper_2607_15413_gb300 import fsz
    sizes = [int(v) for v in lines["sizes"].split()]
    assert sizes[1] == ctypes.sizeof(fsz.FszCField) == 80
    assert sizes[2] == ctypes.sizeof(fsz.FszDField) == 32
    assert sizes[0] == ctypes.sizeof(fsz.FszDims) == 32
    assert sizes[3] == ctypes.sizeof(fsz.FszSchedule)
    assert sizes[5] == ctypes.sizeof(fsz.FszServerConfig)
    assert sizes[6] == ctypes.sizeof(fsz.FszRequest)
    assert sizes[7] == ctypes.sizeof(fsz.FszCompletion)
    assert sizes[8] == ctypes.sizeof(fsz.FszServerStats)
    eb_off, nb_off, cap_off = (int(v) for v in lines["offsets"].split())
    assert eb_off == fsz.FszCField.eb.offset and nb_off == fsz.FszCField.out_bytes.offset
    assert cap_off == fsz.FszDField.out_capacity_elems.offset
    assert lines["version"] == fsz.fsz_version()
    b1000, b0 = (int(v) for v in lines["bound"].split())
    assert b1000 == fsz.fsz_compress_bound(1000) and b0 == fsz.fsz_compress_bound(0)
    assert int(lines["workspace"]) == fsz.fsz_workspace_bytes(1 << 20)
    assert int(lines["header"]) == fsz.ERR_CORRUPT
    assert [int(v) for v in lines["schedule"].split()] == [0, 0, 0, 2, 2, 4, 16, 4]
    assert int(lines["refused"]) == fsz.ERR_INVALID_ARG
