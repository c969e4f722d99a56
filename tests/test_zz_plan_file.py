"""Plan files: the inputs of a plan in one checked file (Section 4: planning may run on its
own; parameters and (u, v, w) coordinates are read from files).  The format, the checks on
reading and the refusal of damaged files run on the host; one GPU test rebuilds a plan from
its file and compares it with the plan made directly."""
import ctypes as C
import math
import struct

import numpy as np
import pytest

import synth

FNV_OFFSET, FNV_PRIME, MASK = 14695981039346656037, 1099511628211, (1 << 64) - 1


def fnv1a(data: bytes, h: int = FNV_OFFSET) -> int:
    for b in data:
        h = ((h ^ b) * FNV_PRIME) & MASK
    return h


def documented_checksum(body: bytes) -> int:
    # FNV-1a of each 1 MiB block, then FNV-1a over the block digests as 8 little-endian bytes
    digests = [fnv1a(body[i:i + (1 << 20)]) for i in range(0, len(body), 1 << 20)]
    return fnv1a(b"".join(struct.pack("<Q", d) for d in digests))


def _case(m=3000, seed=96):
    import paper_2605_26347_gb300 as pkg
    uvw = np.ascontiguousarray(synth.make_uvw(m, 60, 1.28e9, seed))
    fov = math.radians(1.0)
    params = pkg.default_params(256, 256, fov, fov, n_wbins=3, tile_size=64)
    w = np.random.default_rng(seed).uniform(0.2, 1.5, m).astype(np.float32)
    return pkg, uvw, params, w


def test_round_trip_and_documented_layout(tmp_path, rimo_lib):
    pkg, uvw, params, w = _case(m=50_000)
    path = tmp_path / "a.rimoplan"
    pkg.write_plan_file(str(path), uvw, params, weights=w)
    raw = path.read_bytes()
    psize = C.sizeof(pkg.PlanParams)
    assert raw[:8] == b"RIMOPLAN"
    version, pbytes, M, hw, zero = struct.unpack_from("<IIqII", raw, 8)
    assert (version, pbytes, M, hw, zero) == (1, psize, uvw.shape[0], 1, 0)
    assert len(raw) == 32 + psize + 24 * M + 4 * M + 8
    assert raw[32:32 + psize] == bytes(params)
    assert np.array_equal(np.frombuffer(raw, np.float64, 3 * M, 32 + psize).reshape(M, 3), uvw)
    assert np.array_equal(np.frombuffer(raw, np.float32, M, 32 + psize + 24 * M), w)
    assert len(raw) - 8 > (1 << 20)  # several checksum blocks
    assert struct.unpack_from("<Q", raw, len(raw) - 8)[0] == documented_checksum(raw[:-8])
    p2, M2, has_w = pkg.plan_file_info(str(path))
    assert (M2, has_w) == (uvw.shape[0], True) and bytes(p2) == bytes(params)
    pkg.write_plan_file(str(path), uvw, params)  # replaces the file; no weights
    assert pkg.plan_file_info(str(path))[2] is False


def _damaged(raw: bytes, psize: int):
    M = struct.unpack_from("<q", raw, 16)[0]
    flip = bytearray(raw)
    flip[32 + psize + 24 * (M // 2) + 3] ^= 0x10          # one bit of a coordinate
    bad_sum = bytearray(raw)
    bad_sum[-1] ^= 0x01
    magic = bytearray(raw)
    magic[0:8] = b"NOTAPLAN"
    version = bytearray(raw)
    version[8:12] = struct.pack("<I", 2)
    big_m = bytearray(raw)
    big_m[16:24] = struct.pack("<q", 1 << 40)
    return {"flipped coordinate bit": (bytes(flip), "checksum"),
            "flipped checksum bit": (bytes(bad_sum), "checksum"),
            "truncated": (raw[:-100], "size"),
            "extended": (raw + b"\0" * 16, "size"),
            "foreign magic": (bytes(magic), "not a plan file"),
            "unknown version": (bytes(version), "version"),
            "M out of range": (bytes(big_m), "M out of range"),
            "header only": (raw[:20], "shorter")}


def test_damaged_files_are_refused_before_any_device_work(tmp_path, rimo_lib):
    pkg, uvw, params, w = _case()
    good = tmp_path / "good.rimoplan"
    pkg.write_plan_file(str(good), uvw, params, weights=w)
    raw = good.read_bytes()
    for name, (data, why) in _damaged(raw, C.sizeof(pkg.PlanParams)).items():
        path = tmp_path / "bad.rimoplan"
        path.write_bytes(data)
        with pytest.raises(pkg.RimoError) as e:
            pkg.plan_file_info(str(path))
        assert e.value.status == 1 and why in str(e.value), (name, str(e.value))
        # creation checks the file first, so no GPU is touched and nothing is returned
        out = C.c_void_p(123)
        st = rimo_lib.rimo_plan_create_from_file(str(path).encode(), None, C.byref(out))
        assert st == 1 and out.value is None, name
    with pytest.raises(pkg.RimoError):
        pkg.plan_file_info(str(tmp_path / "missing.rimoplan"))


def test_well_formed_files_with_bad_contents_are_refused(tmp_path, rimo_lib):
    # a valid checksum over contents that plan creation would refuse: the file is checked
    # like the arguments of rimo_plan_create after its checksum
    pkg, uvw, params, w = _case()
    good = tmp_path / "good.rimoplan"
    pkg.write_plan_file(str(good), uvw, params, weights=w)
    raw = bytearray(good.read_bytes())
    psize = C.sizeof(pkg.PlanParams)
    M = uvw.shape[0]
    bad_params = pkg.PlanParams.from_buffer_copy(bytes(raw[32:32 + psize]))
    bad_params.nx = 100
    edits = {"nx and ny": (32, bytes(bad_params)),
             "non-finite": (32 + psize + 24 * 11 + 16, struct.pack("<d", float("nan"))),
             "weights must be": (32 + psize + 24 * M + 4 * 9, struct.pack("<f", -0.5))}
    for why, (off, data) in edits.items():
        buf = bytearray(raw)
        buf[off:off + len(data)] = data
        buf[-8:] = struct.pack("<Q", documented_checksum(bytes(buf[:-8])))
        path = tmp_path / "edited.rimoplan"
        path.write_bytes(bytes(buf))
        with pytest.raises(pkg.RimoError) as e:
            pkg.plan_file_info(str(path))
        assert e.value.status == 1 and why in str(e.value), (why, str(e.value))


def test_write_refuses_what_plan_creation_would(tmp_path, rimo_lib):
    pkg, uvw, params, w = _case()
    path = str(tmp_path / "x.rimoplan")
    bad_uvw = uvw.copy()
    bad_uvw[7, 2] = np.nan
    bad_w = w.copy()
    bad_w[5] = -1.0
    bad_params = pkg.default_params(100, 256, 0.01, 0.01)
    for args, kw in (((bad_uvw, params), {}), ((uvw, params), {"weights": bad_w}), ((uvw, bad_params), {})):
        with pytest.raises(pkg.RimoError) as e:
            pkg.write_plan_file(path, *args, **kw)
        assert e.value.status == 1
    with pytest.raises(pkg.RimoError):
        pkg.write_plan_file(str(tmp_path / "no_such_dir" / "x.rimoplan"), uvw, params)


@pytest.mark.gpu
def test_plan_from_file_is_the_plan_made_directly(tmp_path):
    import torch
    pkg, uvw, params, w = _case()
    path = str(tmp_path / "p.rimoplan")
    pkg.write_plan_file(path, uvw, params, weights=w)
    direct = pkg.Plan(uvw, params)
    direct.set_weights(w)
    loaded = pkg.Plan.from_file(path)
    ws_a, b_a, s_a = direct.bins()
    ws_b, b_b, s_b = loaded.bins()
    assert np.array_equal(ws_a, ws_b) and np.array_equal(b_a, b_b) and np.array_equal(s_a, s_b)
    assert loaded.info()["weighted"] == 1
    x = torch.from_numpy(synth.make_sky(256, 5).astype(np.complex64)).cuda()
    za = direct.phi_adj_phi(x)
    zb = loaded.phi_adj_phi(x)
    torch.cuda.synchronize()
    # fixed-point gridding: the same plan gives the same bits
    assert torch.equal(torch.view_as_real(za), torch.view_as_real(zb))
    direct.close()
    loaded.close()
