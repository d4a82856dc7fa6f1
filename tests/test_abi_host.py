"""Host-side checks (no GPU): the C ABI library builds, loads and exports
every function include/madflow_gb300.h declares; the oracle and the CUDA
path share no source."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "madflow_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2105_10529_gb300 import build, _lib
    build.build()
    L = ctypes.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert sorted(_lib.exported_symbols()) == names
    # the binding declares the same calls
    lib = _lib.lib()
    for n in names:
        assert getattr(lib, n).argtypes is not None or n in ("mf_destroy",)


def test_default_config_and_process_info_without_gpu():
    from paper_2105_10529_gb300 import _lib
    from paper_2105_10529_gb300.api import make_config, process_info
    cfg = make_config()
    assert cfg.mt == 173.0 and cfg.n_bins == 50 and cfg.precision == _lib.MF_MIXED
    assert process_info(_lib.MF_GG_TTGG) == (6, 18)
    assert process_info(_lib.MF_EE_MUMU) == (4, 2)
    assert process_info(_lib.MF_UU_TT) == (4, 10)
    assert process_info(_lib.MF_UG_TTU) == (5, 14)
    assert process_info(_lib.MF_GG_TTGGG) == (7, 22)
    with pytest.raises(_lib.MfError):
        process_info(17)


def test_setters_reject_a_null_context_without_gpu():
    """The context setters check their arguments before touching the device: a null context is
    MF_ERR_ARG (1) for every one of them."""
    from paper_2105_10529_gb300 import _lib
    L = _lib.lib()
    assert L.mf_set_helicity_sampling(None, 4, 0) == 1
    assert L.mf_set_helicity_split(None, 1) == 1
    assert L.mf_set_precision(None, 1) == 1


def test_oracle_and_cuda_path_share_no_code():
    cuda_dir = os.path.join(ROOT, "paper_2105_10529_gb300")
    oracle_dir = os.path.join(ROOT, "oracle")
    for d, _, files in os.walk(cuda_dir):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                txt = open(os.path.join(d, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mf_oracle" not in txt and "or_" + "philox" not in txt, f
    for f in os.listdir(oracle_dir):
        if f.endswith((".c", ".h", ".py")):
            txt = open(os.path.join(oracle_dir, f)).read()
            assert "csrc" not in txt and "madflow_gb300.h" not in txt and "paper_2105_10529_gb300." + "gen" not in txt, f


def test_generated_headers_are_current():
    """The committed generated headers equal the generator's output."""
    from fractions import Fraction
    from paper_2105_10529_gb300.gen import qcd_diagrams as Q
    from paper_2105_10529_gb300.gen.__main__ import PROCESSES, OUT
    for k, name, sym in PROCESSES:
        src, st = Q.generate_gluon_process(k, name, sym)
        assert open(os.path.join(OUT, f"me_{name}.cuh")).read() == src
        assert st["n_diag"] == {2: 3, 3: 16, 4: 123}[k]
        assert st["ncol"] == {2: 2, 3: 6, 4: 24}[k]


def test_missing_library_fails_loudly(tmp_path):
    """Without the built CUDA library every entry point raises; nothing falls
    back to a CPU path (checked in a fresh interpreter whose library path
    points at an empty directory)."""
    import subprocess
    import sys
    code = (
        "import paper_2105_10529_gb300._lib as L\n"
        f"L.LIB_PATH = {str(tmp_path / 'absent.so')!r}\n"
        "from paper_2105_10529_gb300 import inputs as IN\n"
        "from paper_2105_10529_gb300.api import Context, process_info\n"
        "for f in (lambda: process_info(IN.GG_TT), lambda: Context(IN.Physics(), IN.make_pdf_grid())):\n"
        "    try:\n"
        "        f()\n"
        "    except RuntimeError as e:\n"
        "        assert 'no CPU fallback' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('no error without the library')\n"
        "print('ok')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
