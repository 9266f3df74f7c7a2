"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point declared in include/*.h, and its host-only calls (packing,
size queries, schedule validation) behave as documented."""

import glob
import os
import re

import numpy as np
import pytest

import paper_2001_10049_gb300 as dib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(dibella_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(dib.library_path())
    declared = declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    # and the binding wraps each of them under the same name
    for name in declared:
        assert callable(getattr(dib, name)), name


def test_debug_library_exports_the_same_symbols():
    """The bounds-checked build (libdibella_debug.so) is the same C ABI."""
    import ctypes
    from paper_2001_10049_gb300 import _build
    path = _build.build(debug=True)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.dibella_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in lib.dibella_version()


def test_version_and_error_string():
    assert "sm_103a" in dib.dibella_version()
    assert isinstance(dib.dibella_last_error(), str)


def decode_copy(words, start_word, length):
    out = []
    for q in range(length):
        w = int(words[start_word + q // 16])
        out.append("ACGT"[(w >> (2 * (q % 16))) & 3])
    return "".join(out)


def test_pack_layout_round_trip():
    rng = np.random.default_rng(0)
    reads = ["".join(rng.choice(list("ACGT"), size=n)) for n in (0, 1, 15, 16, 17, 63, 64, 65, 1000)]
    reads[3] = reads[3].lower()
    ascii = np.frombuffer("".join(reads).encode(), dtype=np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads]).astype(np.int64)
    words, woffs, lens = dib.dibella_pack_reads(ascii, offs, n_threads=3)
    assert words.dtype == np.uint32 and len(words) == dib.dibella_packed_words(offs)
    assert list(words[:8]) == [0] * 8 and list(words[-8:]) == [0] * 8
    comp = str.maketrans("ACGT", "TGCA")
    for r, s in enumerate(reads):
        s = s.upper()
        assert lens[r] == len(s)
        assert woffs[r] % 4 == 0
        cw = ((len(s) + 15) // 16 + 3) // 4 * 4
        assert decode_copy(words, woffs[r], len(s)) == s
        assert decode_copy(words, woffs[r] + cw, len(s)) == s.translate(comp)[::-1]
        if r + 1 < len(reads):
            assert woffs[r + 1] == woffs[r] + 2 * cw


def test_pack_rejects_non_acgt():
    ascii = np.frombuffer(b"ACGTNACGT", dtype=np.uint8)
    offs = np.array([0, 4, 9], dtype=np.int64)
    with pytest.raises(dib.DibellaError) as e:
        dib.dibella_pack_reads(ascii, offs)
    assert e.value.code == dib.DIBELLA_EBASE and "byte 4" in str(e.value)


def test_size_queries_validate():
    assert dib.dibella_xdrop_workspace_bytes(0, 0) > 0
    a = dib.dibella_xdrop_workspace_bytes(1000, 6000)
    b = dib.dibella_xdrop_workspace_bytes(2000, 6000)
    c = dib.dibella_xdrop_workspace_bytes(1000, 100000)
    assert a < b and a < c
    for bad in ((-1, 10), (10, -1), (10, (1 << 24) + 1)):
        with pytest.raises(dib.DibellaError):
            dib.dibella_xdrop_workspace_bytes(*bad)
    assert dib.dibella_staging_bytes(10) >= 10 * 64
    with pytest.raises(dib.DibellaError):
        dib.dibella_packed_words(np.array([0, 5, 3], dtype=np.int64))


def test_schedule_validation():
    s = dib.dibella_get_default_schedule()
    d = s.as_dict()
    assert d["narrow_band_cap"] in (32, 48, 64) and d["wide_slots"] in (0, 8, 16, 24, 32)
    bad = dib.Schedule.from_dict(dict(d, narrow_band_cap=40))
    with pytest.raises(dib.DibellaError):
        dib.dibella_set_default_schedule(bad)
    bad = dib.Schedule.from_dict(dict(d, n_buckets=0))
    with pytest.raises(dib.DibellaError):
        dib.dibella_set_default_schedule(bad)
    dib.dibella_set_default_schedule(s)  # the default itself is valid
    assert dib.dibella_get_default_schedule().as_dict() == d


def test_batch_argument_errors_are_synchronous():
    """Bad scalars are refused before any device work (no GPU touched)."""
    good = dib.Scoring(1, -1, -1, 7)
    bad_scorings = [dib.Scoring(0, -1, -1, 7), dib.Scoring(1, 1, -1, 7), dib.Scoring(1, -1, 0, 7),
                    dib.Scoring(1, -1, -1, -1), dib.Scoring(1, -1, -1, (1 << 30) + 1),
                    dib.Scoring(65, -1, -1, 7)]
    for sc in bad_scorings:
        with pytest.raises(dib.DibellaError) as e:
            dib.dibella_xdrop_batch(0, 0, 0, 0, 0, 0, 17, sc, 0, 0, 0, stream=0)
        assert e.value.code == dib.DIBELLA_EINVAL
    for k in (0, 33):
        with pytest.raises(dib.DibellaError):
            dib.dibella_xdrop_batch(0, 0, 0, 0, 0, 0, k, good, 0, 0, 0, stream=0)
    with pytest.raises(dib.DibellaError):  # null workspace
        dib.dibella_xdrop_batch(0, 0, 0, 0, 0, 0, 17, good, 0, 0, 0, stream=0)
    with pytest.raises(dib.DibellaError):  # misaligned workspace
        dib.dibella_xdrop_batch(0, 0, 0, 0, 0, 0, 17, good, 0, 4096 + 8, 1 << 20, stream=0)
