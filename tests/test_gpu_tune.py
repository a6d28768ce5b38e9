"""The tile-configuration autotuner: its choice, the certificates after tuning, its table file."""
import json

import numpy as np
import pytest

from gpu_helpers import assert_cert_parity
from oracle import adagio as O
from oracle.certificate import certificate
from paper_1609_05388_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    wl = synth.mnist_like(seed=1, n=5000)
    f = O.fit(wl.X.astype(np.float64), 150, 3)
    Y = O.embed(f.A, wl.X).astype(np.float32)
    return wl.X, Y


def test_autotune_choice_and_certificates_after_it(data, tmp_path):
    from paper_1609_05388_gb300 import adagio as lib
    X, Y = data
    n = X.shape[0]
    with lib.Context(0) as ctx:
        best = ctx.autotune_tiles(X, Y, 0.1, precision=lib.PREC_FP16X3)
        assert best["variant"] in (lib.TILES_SINGLE, lib.TILES_PAIR)
        assert best["band"] in (4, 8, 16, 32, 64) and best["tile_ms"] > 0.0
        T = -(-n // 256) * 2
        assert best["size_class"] == int(np.ceil(np.log2(T)))
        # later certificates of this size class use the tuned configuration
        assert ctx.tile_kernel_for(n) == best["variant"]
        o = certificate(X, Y, 0.1)
        g = ctx.distortion(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), 0.1)
        assert_cert_parity(g, o, X, Y)
        path = str(tmp_path / "tiles.json")
        ctx.tune_save(path)
    table = json.load(open(path))
    assert table["entries"][0]["variant"] == best["variant"]
    with lib.Context(0) as ctx2:
        assert ctx2.tile_kernel_for(n) == lib.TILES_SINGLE
        ctx2.tune_load(path)
        assert ctx2.tile_kernel_for(n) == best["variant"]


def test_tile_table_of_another_device_or_malformed_is_rejected(tmp_path):
    from paper_1609_05388_gb300 import adagio as lib
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"device": "some other GPU", "entries": [
        {"size_class": 5, "variant": 2, "band": 4, "tile_ms": 1.0}]}))
    bad = tmp_path / "bad.json"
    bad.write_text('{"device": "x", "entries": [{"size_class": 5, "variant": 7}]}')
    with lib.Context(0) as ctx:
        for p in (other, bad, tmp_path / "missing.json"):
            with pytest.raises(lib.AdagioError) as ei:
                ctx.tune_load(str(p))
            assert ei.value.code == lib.E_INVALID_ARG
        with pytest.raises(lib.AdagioError):
            ctx.set_tile_kernel(lib.TILES_SINGLE, 65)
