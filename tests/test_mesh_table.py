"""The library's marching-cubes case table (built on the host from the face
rule, no GPU needed) against the oracle's per-cell face walk, all 256 cases."""
import os
import shutil

import pytest

from oracle import mesh as m


@pytest.fixture(scope="module")
def table():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2308_13175_gb300 import binding, build
    build.build()
    return binding.gp_mesh_case_table()


def test_case_table_matches_the_oracle(table):
    ntri, edges = table
    for case in range(256):
        want = m.case_triangles(case)
        assert int(ntri[case]) == len(want), case
        got = [tuple(int(e) for e in edges[case, 3 * k:3 * k + 3]) for k in range(len(want))]
        assert got == list(want), case
        assert all(int(e) == 255 for e in edges[case, 3 * len(want):])
