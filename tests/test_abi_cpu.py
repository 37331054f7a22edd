"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
entry point include/stereovae.h declares, and its host-only functions behave."""
import ctypes
import os
import re

import pytest

from paper_2305_11566_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"SV_API[^;(]*?\b(sv_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("sv_create", "sv_coarse_match", "sv_refine", "sv_pipeline", "sv_refine_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(svlib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(svlib, n), n
        assert n in binding.API, n


def test_param_count_matches_layout(svlib):
    assert binding.param_count(synth.NET_SMALL, 7) == 91921 == synth.NET_SMALL.n_params()
    assert binding.param_count(synth.NET_WIDE, 9) == 366113 == synth.NET_WIDE.n_params()


def test_invalid_configs_rejected(svlib):
    bad = []
    c = binding.make_config(synth.NET_SMALL, 8)       # even window
    bad.append(c)
    c = binding.make_config(synth.NET_SMALL, 17)      # too large
    bad.append(c)
    c = binding.make_config(synth.NetShape((16, 24, 64), 64, (64, 32, 16)), 7)  # width not /16
    bad.append(c)
    c = binding.make_config(synth.NET_SMALL, 7, 5)    # precision
    bad.append(c)
    c = binding.make_config(synth.NET_SMALL, 7, "fp8")  # FP8: a 16-wide input to a tensor-core layer
    bad.append(c)
    c = binding.make_config(synth.NetShape((32, 64, 128), 128, (48, 64, 32)), 7, "fp8")  # dec1 width 48
    bad.append(c)
    for c in bad:
        assert svlib.sv_param_count(ctypes.byref(c)) == 0
        h = ctypes.c_void_p()
        assert svlib.sv_create(ctypes.byref(c), 0, ctypes.byref(h)) == binding.SV_ERR_INVALID_ARG
        assert not h.value


def test_fp8_config_accepted(svlib):
    # widths that are multiples of 32 where a quantised layer reads them (dec2's and dec3's
    # outputs feed BF16 layers and may be 16 wide)
    for shape in (synth.NET_WIDE, synth.NetShape((32, 64, 128), 128, (128, 48, 16))):
        c = binding.make_config(shape, 9, "fp8")
        assert svlib.sv_param_count(ctypes.byref(c)) == shape.n_params()


def test_status_strings(svlib):
    for i, n in enumerate(["SV_OK", "SV_ERR_INVALID_ARG", "SV_ERR_CUDA", "SV_ERR_OOM", "SV_ERR_UNSUPPORTED",
                           "SV_ERR_TIMEOUT", "SV_ERR_STATE"]):
        assert svlib.sv_status_string(i).decode() == n
    assert svlib.sv_last_error(None).decode() == "NULL context"


def test_null_context_calls_rejected(svlib):
    assert svlib.sv_destroy(None) == binding.SV_ERR_INVALID_ARG
    assert svlib.sv_coarse_match(None, None, 0, None, None, None, None) == binding.SV_ERR_INVALID_ARG
    assert svlib.sv_refine(None, None, None, 0, None, None) == binding.SV_ERR_INVALID_ARG
    assert svlib.sv_pipeline(None, None, 0, None, None) == binding.SV_ERR_INVALID_ARG
    assert svlib.sv_refine_backward(None, None, None, None, None, None, None) == binding.SV_ERR_INVALID_ARG


def test_create_without_device_fails_cleanly(svlib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = binding.make_config(synth.NET_SMALL, 7)
    h = ctypes.c_void_p()
    assert svlib.sv_create(ctypes.byref(c), 0, ctypes.byref(h)) == binding.SV_ERR_CUDA
    assert not h.value


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI's structs have the C compiler's sizes and offsets."""
    import subprocess
    fields = {"sv_pair": (binding.SvPair, ["left", "right", "width", "height", "pitch", "max_disp"]),
              "sv_config": (binding.SvConfig, ["window", "enc_ch", "latent_ch", "dec_ch", "precision", "flags"]),
              "sv_coarse_opts": (binding.SvCoarseOpts, [f for f, _ in binding.SvCoarseOpts._fields_])}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "stereovae.h"', "int main(void) {"]
    for st, (_, names) in fields.items():
        src.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for n in names:
            src.append(f'  printf("{st}.{n} %zu\\n", offsetof({st}, {n}));')
    src.append("  return 0;\n}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, (cls, names) in fields.items():
        assert int(got[st]) == ctypes.sizeof(cls), st
        for n in names:
            assert int(got[f"{st}.{n}"]) == getattr(cls, n).offset, (st, n)


def test_pair_array_marshalling():
    """The pair array handed to the C ABI (one numpy buffer over the sv_pair layout) holds the
    same bytes as sv_pair structs built field by field, and follows a pair whose image is
    replaced (the cached fields are dropped on any attribute change)."""
    import torch
    imgs = [torch.zeros((8 + i, 32 + 16 * (i % 3)), dtype=torch.uint8) for i in range(5)]
    dps = [binding.DevicePair(imgs[i], imgs[(i + 1) % 5], 30 + i, 8 + i, 20 + i) for i in range(5)]
    arr = binding._pairs_array(dps)
    ref = (binding.SvPair * 5)(*[binding.SvPair(p.left.data_ptr(), p.right.data_ptr(), p.width, p.height,
                                                 int(p.left.stride(0)), p.max_disp) for p in dps])
    assert bytes(memoryview(arr)) == bytes(memoryview(ref))
    dps[2].left = imgs[4]
    dps[2].max_disp = 7
    arr = binding._pairs_array(dps)
    assert arr[2].left == imgs[4].data_ptr() and arr[2].max_disp == 7 and arr[2].pitch == imgs[4].stride(0)
    assert len(binding._pairs_array([])) == 1  # a one-element placeholder for empty calls
