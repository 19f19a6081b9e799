"""CPU checks of the boundary: the library builds, loads and exports every
function include/hecnn.h declares; host-side parameter logic matches the
oracle (no GPU calls)."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import ckks, gaussian
from paper_2102_00319_gb300 import build as B
from paper_2102_00319_gb300 import hecnn as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return H.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "hecnn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    declared = header_functions()
    assert len(declared) >= 40
    out = subprocess.check_output(["nm", "-D", "--defined-only", H.LIB_PATH]).decode()
    exported = set(re.findall(r" T (hc_[a-z0-9_]+)", out))
    assert set(declared) <= exported, sorted(set(declared) - exported)
    assert set(declared) == set(H.EXPORTS)


def test_library_links_no_oracle():
    out = subprocess.check_output(["nm", "-D", H.LIB_PATH]).decode()
    assert not re.search(r"\bor_[a-z]", out)


@pytest.mark.parametrize("log_n,q_bits,p_bits", [
    (12, [50, 30, 30], [50]),
    (14, [60] + [40] * 6, [60]),
    (16, [60] + [50] * 20, [60] * 7),
    (10, [30, 25, 25], [30, 30]),
    (10, [30] * 56, [30] * 8),     # the longest chain the library accepts (64 primes)
    (11, [61, 61, 61], [61, 61]),  # the widest primes
])
def test_prime_chain_matches_oracle(lib, log_n, q_bits, p_bits):
    p = H.hc_params_create(log_n, q_bits, p_bits, 30)
    op = ckks.Params(log_n, q_bits, p_bits, 30)
    assert H.hc_params_primes(p) == op.chain
    n, L, alpha, dnum = H.hc_params_info(p)
    assert (n, L, alpha, dnum) == (op.N, op.L, op.alpha, op.dnum)


@pytest.mark.parametrize("sigma", [3.2, 1.0, 2.5, 4.75, 6.0])
def test_gaussian_table_matches_oracle(lib, sigma):
    p = H.hc_params_create(10, [40], [40], 20, sigma)
    assert H.hc_params_cdt(p) == [int(v) for v in gaussian.cdt_table(sigma)]


def test_bad_parameters_rejected(lib):
    for args in ((9, [40], [40]), (12, [70], [40]), (12, [40], []), (10, [20] * 60, [20] * 10)):
        with pytest.raises(H.HcError) as e:
            H.hc_params_create(args[0], args[1], args[2], 20)
        assert e.value.code == -1
