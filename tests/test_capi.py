"""CPU-only checks of the C ABI: the library loads without a GPU, exports every
entry point include/phe.h declares, and rejects bad parameter sets on the host
before any CUDA call."""
import ctypes
import os
import re

import pytest

import synth
from paper_2505_07329_b300 import build, phe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(testing=None):
    """Function names include/*.h declares: testing=None all of them, True
    those inside #ifdef PHE_TESTING blocks, False the others."""
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            test_blocks = re.findall(r"#ifdef PHE_TESTING(.*?)#endif", text, flags=re.S)
            prod = re.sub(r"#ifdef PHE_TESTING.*?#endif", "", text, flags=re.S)
            pat = r"^[A-Za-z_][\w\s\*]*?\b(phe_\w+)\s*\("
            if testing is not True:
                names |= set(re.findall(pat, prod, flags=re.M))
            if testing is not False:
                for b in test_blocks:
                    names |= set(re.findall(pat, b, flags=re.M))
    return names


@pytest.fixture(scope="module")
def L():
    build.build()
    return phe.lib()


def test_library_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(L, n), f"{phe.TEST_LIB_PATH} does not export {n}"


def test_production_library_exports_no_secret_key_call():
    # the server never holds the key (Sec. 5): libphe.so exports every
    # production call and none of the client-side ones
    build.build()
    prod = ctypes.CDLL(phe.LIB_PATH)
    for n in sorted(header_functions(testing=False)):
        assert hasattr(prod, n), f"libphe.so does not export {n}"
    test_only = header_functions(testing=True)
    assert test_only == set(phe.TEST_ONLY)
    for n in sorted(test_only):
        assert not hasattr(prod, n), f"libphe.so exports the client-side call {n}"
    tl = ctypes.CDLL(phe.TEST_LIB_PATH)
    for n in sorted(test_only):
        assert hasattr(tl, n), f"libphe_test.so does not export {n}"


def test_test_keygen_rejects_null_arguments(L):
    assert L.phe_test_keygen(None, 1, 1, None) == phe.PHE_EINVAL


def test_binding_covers_the_header():
    assert set(phe.SIGNATURES) == header_functions()


def test_status_strings(L):
    for code, name in enumerate(["PHE_OK", "PHE_EINVAL", "PHE_ENOMEM", "PHE_EBUSY", "PHE_ETIMEOUT",
                                 "PHE_ECUDA", "PHE_EUNSUPPORTED"]):
        assert phe.phe_status_string(code) == name


@pytest.mark.parametrize("N,q,k,msg", [
    (1000, synth.Q60, 32, "power of two"),
    (128, synth.Q60, 32, "power of two"),
    (16384, synth.Q60, 32, "power of two"),
    (4096, synth.Q60 + 2, 32, "not 1 mod 2N"),
    (4096, (1 << 60) + 8193 * 2, 32, "not 1 mod"),
    (4096, 1 + 8192 * 3 * (2 ** 50 // 8192) * 8, 32, "not prime"),
    (4096, (1 << 52) + 1, 32, "2^53 < q"),
    (4096, synth.Q60, 0, "log2_qout"),
    (4096, synth.Q60, 33, "log2_qout"),
])
def test_ctx_create_rejects_bad_parameters(L, N, q, k, msg):
    with pytest.raises(phe.PheError) as ei:
        phe.phe_ctx_create(N, q, k, 0)
    assert ei.value.status == phe.PHE_EINVAL
    assert msg in str(ei.value)


def test_null_arguments_are_rejected(L):
    assert L.phe_ctx_create(None, 0, None) == phe.PHE_EINVAL
    assert L.phe_matmul(None, None, 0, 1, None, None, None, None, 0, None) == phe.PHE_EINVAL
    assert L.phe_modswitch(None, None, None, 0, None) == phe.PHE_EINVAL
    assert L.phe_weights_upload(None, None, 1, 1, 1, None, None) == phe.PHE_EINVAL
    assert phe.phe_weights_device_bytes(None) == 0
    assert L.phe_ksk_upload(None, None, None, 0, 26, 1, None) == phe.PHE_EINVAL
    assert L.phe_pack(None, None, 1, 1, None, None, None, None, 0, None) == phe.PHE_EINVAL
    assert L.phe_matmul_packed(None, None, None, 0, 1, None, None, None, None, 0, None) == phe.PHE_EINVAL
    assert phe.phe_ksk_device_bytes(None) == 0
    L.phe_ctx_destroy(None)
    L.phe_weights_free(None)
    L.phe_ksk_free(None)


@pytest.mark.parametrize("q,rns,msg", [
    (synth.Q_RNS + 16384, (synth.RNS_P1, synth.RNS_P2), "q = p1 * p2"),
    (synth.Q_RNS, (synth.RNS_P1, synth.RNS_P1), "distinct"),
    (synth.RNS_P1 * 1073709057, (synth.RNS_P1, 1073709057), "p1 and p2 must be prime"),
    (synth.Q_RNS, None, "not prime"),
])
def test_rns_modulus_is_validated(L, q, rns, msg):
    import sympy
    assert sympy.isprime(synth.RNS_P1) and sympy.isprime(synth.RNS_P2)
    with pytest.raises(phe.PheError) as ei:
        phe.phe_ctx_create(4096, q, 32, 0, rns=rns)
    assert ei.value.status == phe.PHE_EINVAL
    assert msg in str(ei.value)


@pytest.mark.parametrize("N,q,k,rns,flags,msg", [
    (2048, 1 << 39, 26, None, 0, "needs rns_p1"),
    (2048, 1 << 39, 39, (synth.RNS_P1, synth.RNS_P2), 0, "log2_qout"),
    (2048, 1 << 39, 26, (synth.RNS_P1, synth.RNS_P2), 1, "no 64-bit form"),
    (2048, 1 << 45, 26, (synth.RNS_P1, synth.RNS_P2), 0, "exact products"),
    (2048, 1 << 4, 2, (synth.RNS_P1, synth.RNS_P2), 0, "8 <= k"),
])
def test_power_of_two_modulus_is_validated(L, N, q, k, rns, flags, msg):
    """q = 2^K (the paper's parameter set) runs through p1 p2 and needs the
    exact-range condition N * 127 * 2^(K-1) < p1 p2 / 2 (2^45 at N = 2048
    breaks it; 2^39 keeps it with L up to 4)."""
    with pytest.raises(phe.PheError) as ei:
        phe.phe_ctx_create(N, q, k, 0, rns=rns, flags=flags)
    assert ei.value.status == phe.PHE_EINVAL
    assert msg in str(ei.value)


@pytest.mark.parametrize("N,rows,T,flags,want", [
    (4096, 2048, 16, 0, (16, 1)),                   # one token per RLWE (Eq. (pack_rotate) per token)
    (4096, 8192, 3, 0, (6, 1)),                     # two RLWEs per token
    (4096, 2048, 16, phe.PHE_PACK_DENSE, (8, 2)),   # dense: 2 tokens fill the ring
    (4096, 512, 17, phe.PHE_PACK_DENSE, (3, 8)),    # 8 per RLWE, the last holds 1
    (4096, 700, 12, phe.PHE_PACK_DENSE, (3, 5)),    # 5 x 700 = 3500 of 4096 coefficients
    (4096, 2049, 5, phe.PHE_PACK_DENSE, (5, 1)),    # above N/2: unchanged
    (4096, 8192, 3, phe.PHE_PACK_DENSE | phe.PHE_OUT_RAW, (6, 1)),
    (256, 1, 300, phe.PHE_PACK_DENSE, (2, 256)),
    (4096, 512, 0, phe.PHE_PACK_DENSE, (0, 8)),
])
def test_pack_layout(L, N, rows, T, flags, want):
    assert phe.phe_pack_layout(N, rows, T, flags) == want


@pytest.mark.parametrize("N,rows,flags", [(4096, 0, 0), (3000, 10, 0), (4096, 10, 4), (0, 10, 0)])
def test_pack_layout_rejects_bad_arguments(L, N, rows, flags):
    with pytest.raises(phe.PheError) as ei:
        phe.phe_pack_layout(N, rows, 4, flags)
    assert ei.value.status == phe.PHE_EINVAL
