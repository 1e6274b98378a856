"""The network checkpoint format of cnn_save / cnn_load (include/helm.h), checked on
the CPU: cnn_load validates the whole file on the host (magic, version, the
architecture against the parameter count, the payload length and its FNV-1a
checksum) before it touches the device, so every malformed file is refused with
HELM_EINVAL without a GPU.  The round trip of a real network is a GPU test."""
import struct

import numpy as np
import pytest

from oracle import cnn


@pytest.fixture(scope="module")
def n():
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native
    return native


def _fnv1a(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _file(widths=(16, 32), nparams=None, magic=b"HELMCNN1", version=1, payload=None, checksum=None, flags=0):
    specs = cnn.layer_specs(widths=widths)
    npar = cnn.n_params(specs) if nparams is None else nparams
    body = np.arange(npar, dtype=np.float32).tobytes() if payload is None else payload
    ck = _fnv1a(body) if checksum is None else checksum
    w8 = list(widths) + [0] * (8 - len(widths))
    head = magic + struct.pack("<II8IqqIIQ", version, len(widths), *w8, npar, 0, flags, 0, ck)
    return head + body


def _expect_einval(n, path):
    with pytest.raises(n.HelmError) as e:
        n.cnn_load(str(path))
    assert e.value.status == n.HELM_EINVAL
    return str(e.value)


def test_header_layout_is_the_documented_one():
    # magic 8 + version 4 + levels 4 + widths 32 + nparams 8 + adam steps 8 + flags 4 + loss 4 + checksum 8
    assert len(_file(payload=b"")) == 80


def test_malformed_checkpoints_are_refused_on_the_host(n, tmp_path):
    good = _file()
    p = tmp_path / "x.ckpt"
    assert "cannot open" in _expect_einval(n, tmp_path / "missing.ckpt")
    p.write_bytes(_file(magic=b"NOTACKPT"))
    assert "not a network checkpoint" in _expect_einval(n, p)
    p.write_bytes(_file(version=2))
    _expect_einval(n, p)
    p.write_bytes(good[:-4])                                  # truncated payload
    assert "truncated or corrupted" in _expect_einval(n, p)
    p.write_bytes(good + b"\0")                               # trailing bytes
    assert "truncated or corrupted" in _expect_einval(n, p)
    bad = bytearray(good)
    bad[100] ^= 1                                             # one flipped bit in the payload
    p.write_bytes(bytes(bad))
    assert "truncated or corrupted" in _expect_einval(n, p)
    p.write_bytes(_file(nparams=cnn.n_params(cnn.layer_specs(widths=(16, 32))) + 1))
    assert "architecture" in _expect_einval(n, p)
    p.write_bytes(_file(widths=(16, 24)))                     # widths must be multiples of 16
    _expect_einval(n, p)
    p.write_bytes(_file(flags=2))                             # unknown flag bits
    _expect_einval(n, p)
