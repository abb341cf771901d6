"""The C-ABI library loads and exports every entry point include/lloid.h
declares, and the ctypes structures match the C layout (checked against gcc).
No compute call is made: these run without a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lloid.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_04730_b300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"LLOID_API\s+[\w\s\*]+?\b(lloid_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lloid_create", "lloid_load_bank", "lloid_push_strain", "lloid_pull_triggers", "lloid_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2511_04730_b300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in bound, f"{name} has no ctypes signature"


def test_struct_layout_matches_c(lib):
    from paper_2511_04730_b300 import _lib
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lloid.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("lloid_config %zu\nlloid_slice %zu\nlloid_bank_desc %zu\nlloid_trigger %zu\nlloid_event %zu\n",
         sizeof(lloid_config), sizeof(lloid_slice), sizeof(lloid_bank_desc), sizeof(lloid_trigger),
         sizeof(lloid_event));
  P(lloid_config, max_block) P(lloid_config, hbm_budget_bytes) P(lloid_config, cuda_stream) P(lloid_config, flags)
  P(lloid_config, coinc_window) P(lloid_config, form_ratio) P(lloid_config, fir_ctas)
  printf("lloid_tuning %zu\n", sizeof(lloid_tuning));
  P(lloid_tuning, ms) P(lloid_tuning, cand_ratio) P(lloid_tuning, cand_ctas)
  P(lloid_slice, j_start) P(lloid_slice, bases) P(lloid_slice, coeffs)
  P(lloid_bank_desc, ac_half) P(lloid_bank_desc, autocorr)
  P(lloid_trigger, window) P(lloid_trigger, sample) P(lloid_trigger, snr) P(lloid_trigger, im) P(lloid_trigger, xi2)
  P(lloid_event, window) P(lloid_event, net_snr) P(lloid_event, ref_sample)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    m = {"lloid_config": _lib.LloidConfig, "lloid_slice": _lib.LloidSlice, "lloid_tuning": _lib.LloidTuning,
         "lloid_bank_desc": _lib.LloidBankDesc, "lloid_trigger": _lib.LloidTrigger, "lloid_event": _lib.LloidEvent}
    for k, v in got.items():
        if "." in k:
            t, f = k.split(".")
            assert getattr(m[t], f).offset == int(v), k
        else:
            assert ctypes.sizeof(m[k]) == int(v), k


def test_host_only_calls(lib):
    from paper_2511_04730_b300 import _lib
    cfg = _lib.LloidConfig()
    lib.lloid_config_default(ctypes.byref(cfg))
    # the paper's constants (Section II.C.2, II.D.1)
    assert (cfg.f0, cfg.n_down, cfg.n_up, cfg.window_samples) == (2048, 32, 8, 2048)
    # coincidence window: maximum light travel time plus buffer (Section II.D.3), at 2048 Hz
    assert cfg.coinc_window == int((0.0273 + 0.005) * 2048)
    assert cfg.snr_threshold == 4.0 and cfg.window_overlap == 0
    assert cfg.form_ratio == 1.0 and cfg.fir_ctas == 0
    assert lib.lloid_strerror(-4) == b"discontinuous push (t0 is not the stream end)"
    assert lib.lloid_strerror(0) == b"ok"
    assert lib.lloid_last_error(None) == b"null context"


def test_create_rejects_pushes_of_more_than_16_windows(lib):
    """Configuration checks run before any device call: a push that could
    complete 17 one-second windows is refused with LLOID_EINVAL."""
    from paper_2511_04730_b300 import _lib
    cfg = _lib.LloidConfig()
    lib.lloid_config_default(ctypes.byref(cfg))
    cfg.max_block = 16 * cfg.window_samples
    h = ctypes.c_void_p()
    assert lib.lloid_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert not h.value


@pytest.mark.parametrize("rate_in,rate_out,n_fft,z_pad", [
    (16384, 512, 1 << 20, 1 << 18),      # N_out = 32768: one transform no longer fits shared memory
    (1 << 14, 1, 1 << 16, 1 << 14),      # R = 16384 > 4096 polyphase components
    (16384, 2048, 65536, 32768),         # Z = N / 2: no hop
    (16384, 2048, 65536 + 8, 16384),     # N not a power of two
])
def test_whitener_create_rejects_unsupported_sizes(lib, rate_in, rate_out, n_fft, z_pad):
    """The whitener's size checks run before any device call: its own FFTs take
    N_out = n_fft rate_out / rate_in of 4 .. 16384, at most 4096 polyphase
    components and n_fft <= 2^24; the rest is refused with LLOID_EINVAL."""
    from paper_2511_04730_b300 import _lib
    cfg = _lib.LloidWhitenerConfig()
    lib.lloid_whitener_config_default(ctypes.byref(cfg))
    assert (cfg.rate_in, cfg.rate_out, cfg.n_fft, cfg.z_pad, cfg.n_med) == (16384, 2048, 65536, 16384, 7)
    cfg.rate_in, cfg.rate_out, cfg.n_fft, cfg.z_pad = rate_in, rate_out, n_fft, z_pad
    cfg.max_push = 4 * (n_fft // 2 - z_pad) if n_fft // 2 > z_pad else n_fft
    h = ctypes.c_void_p()
    assert lib.lloid_whitener_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert not h.value


def test_product_path_has_no_oracle_import():
    """The product package never imports the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2511_04730_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2511_04730_b300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved
