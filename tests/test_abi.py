"""The C-ABI library builds, loads and exports every symbol include/chebfd.h
declares; host-only entry points agree with the oracle (no GPU needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1510_04895_gb300 import _lib
    return _lib


def declared_functions():
    text = open(os.path.join(ROOT, "include", "chebfd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chebfd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["chebfd_scale_bounds", "chebfd_window_coeffs", "chebfd_filter_block"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    so = built.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (chebfd_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = built.lib()
    for n in declared_functions():
        getattr(L, n)
    assert L.chebfd_abi_version() == 3


def test_binding_covers_every_symbol(built):
    assert set(declared_functions()) <= set(built.SIGNATURES)


@pytest.mark.parametrize("kernel", ["none", "fejer", "jackson", "lanczos"])
def test_window_coeffs_host_entry_matches_oracle(built, kernel):
    from oracle import coeffs
    for (a, b, lo, hi, Np) in [(-4.1, 4.1, -0.1, 0.1, 200), (-5.5, 5.5, -0.06, 0.06, 1438),
                               (-1.0, 3.0, 0.2, 0.9, 37)]:
        got = built.chebfd_window_coeffs(a, b, lo, hi, Np, kernel, 2.0)
        ref = coeffs.filter_coeffs(a, b, lo, hi, Np, kernel, 2.0)
        assert np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()) * 10


def test_invalid_arguments_are_reported(built):
    with pytest.raises(built.ChebFDError) as e:
        built.chebfd_window_coeffs(1.0, -1.0, -0.1, 0.1, 10)
    assert e.value.status == 1 and "b > a" in str(e.value)
    with pytest.raises(built.ChebFDError):
        built.chebfd_window_coeffs(-1.0, 1.0, -0.1, 0.1, 10, kernel=17)


C_PROGRAM = r"""
#include <stdio.h>
#include "chebfd.h"

int main(void) {
    double gc[41];
    chebfd_status st;
    int k;
    if (chebfd_abi_version() != CHEBFD_ABI_VERSION) return 2;
    st = chebfd_window_coeffs(-2.0, 3.0, -0.3, 0.4, 40, CHEBFD_KERNEL_JACKSON, 2.0, gc);
    if (st != CHEBFD_OK) return 3;
    for (k = 0; k <= 40; ++k) printf("%.17g\n", gc[k]);
    st = chebfd_window_coeffs(1.0, -1.0, -0.1, 0.1, 10, CHEBFD_KERNEL_LANCZOS, 2.0, gc);
    printf("%d %s | %s\n", (int)st, chebfd_status_string(st), chebfd_last_error());
    return 0;
}
"""


def test_header_compiles_as_c99_and_links(built, tmp_path):
    """A plain C99 program (-Wall -Werror -pedantic) includes chebfd.h, links
    libchebfd.so and calls host-only entry points: the coefficients match the
    oracle, an invalid call returns EINVAL with a message."""
    from oracle import coeffs
    src = tmp_path / "use_chebfd.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_chebfd"
    libdir = os.path.dirname(built.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lchebfd", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = out.strip().splitlines()
    got = np.array([float(x) for x in lines[:41]])
    ref = coeffs.filter_coeffs(-2.0, 3.0, -0.3, 0.4, 40, "jackson")
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max() * 10
    assert lines[41].startswith("1 ") and "b > a" in lines[41]
