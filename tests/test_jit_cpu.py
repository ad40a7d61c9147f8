"""Segment compiler checks that need no GPU: the generated straight-line
kernels compile with NVRTC for sm_103a for every gate class and arithmetic,
structures are shared across angles, and arguments are validated."""
import pytest

import paper_2508_13615_gb300 as L
import workloads as W

ARITHS = [("c128", L.LQS_ARITH_DF), ("c128", L.LQS_ARITH_F64), ("c64", L.LQS_ARITH_AUTO)]


@pytest.mark.parametrize("dtype,arith", ARITHS)
def test_every_gate_class_compiles(dtype, arith):
    """Random circuits over the whole gate set, with controls landing on
    register slots, thread bits and qubits outside the tile."""
    before = L.lqs_jit_info()
    n = 14 if dtype == "c128" else 15
    total = 0
    for seed in (3, 4):
        c = W.random_circuit(n, 90, seed=seed)
        total += L.lqs_jit_precompile(n, dtype, c.ops, c.params, arith)
    after = L.lqs_jit_info()
    assert after["failed"] == before["failed"], after["last_error"]
    assert after["cached"] >= before["cached"]
    assert total >= 0


def test_angles_do_not_change_the_structure():
    """Coefficients are kernel parameters: a circuit that differs only in its
    angles needs no new kernel."""
    a, b = W.ansatz(22, 2, 5), W.ansatz(22, 2, 6)
    assert list(a.params) != list(b.params)
    first = L.lqs_jit_precompile(22, "c128", a.ops, a.params, L.LQS_ARITH_DF)
    assert first >= 1
    cached = L.lqs_jit_info()["cached"]
    assert L.lqs_jit_precompile(22, "c128", b.ops, b.params, L.LQS_ARITH_DF) == 0
    assert L.lqs_jit_info()["cached"] == cached


def test_modes_and_arguments():
    old = L.lqs_jit_info()["mode"]
    try:
        for m in (L.LQS_JIT_OFF, L.LQS_JIT_ON, L.LQS_JIT_AUTO):
            L.lqs_set_jit(m)
            assert L.lqs_jit_info()["mode"] == m
        with pytest.raises(L.LqsError) as e:
            L.lqs_set_jit(7)
        assert e.value.code == L.lqs.LQS_ERR_ARG
    finally:
        L.lqs_set_jit(old)
    c = W.ansatz(14, 1, 1)
    for bad in (dict(n_qubits=0), dict(n_qubits=40), dict(dtype=5), dict(arith=9)):
        kw = dict(n_qubits=14, dtype="c128", arith=L.LQS_ARITH_DF)
        kw.update(bad)
        with pytest.raises((L.LqsError, ValueError)):
            L.lqs_jit_precompile(kw["n_qubits"], kw["dtype"], c.ops, c.params, kw["arith"])


def test_small_states_have_no_segments_to_compile():
    """States that fit one tile never use the register-tile kernel."""
    c = W.ansatz(8, 3, 2)
    assert L.lqs_jit_precompile(8, "c128", c.ops, c.params, L.LQS_ARITH_DF) == 0


def test_named_barriers_are_never_shared(tmp_path, monkeypatch):
    """Generated kernels give every group barrier of a tile iteration ids of
    its own (a warp may reach a later exchange while another group is still
    at an earlier one); ids are reused only after a block-wide barrier."""
    import glob
    import re
    monkeypatch.setenv("LQS_JIT_DUMP", str(tmp_path))
    for dtype, arith, n in (("c128", L.LQS_ARITH_DF, 19), ("c64", L.LQS_ARITH_AUTO, 19)):
        for seed in (61, 62):
            c = W.random_circuit(n, 160, seed=seed)
            L.lqs_jit_precompile(n, dtype, c.ops, c.params, arith)
        c = W.random_circuit(n, 80, seed=63)
        L.lqs_jit_precompile_adjoint(n, dtype, c.ops, c.params, arith)
    files = glob.glob(str(tmp_path / "*.cu"))
    assert files
    groups = 0
    assert any("lqs_adj_" in f for f in files) and any("lqs_seg_" in f for f in files)
    for f in files:
        src = open(f).read()
        nthreads = int(re.search(r"__launch_bounds__\((\d+),", src).group(1))
        body = re.split(r"for \(; t < G\.ntiles; t \+= [^)]*\) \{", src, maxsplit=1)[1]
        used = set()
        for line in body.splitlines():
            if "__syncthreads" in line:
                used = set()
            m = re.search(r"bar_group\((\d+)u(.*), (\d+)u\);", line)
            if m:
                groups += 1
                ids = set(range(int(m.group(1)), int(m.group(1)) + (1 << m.group(2).count("tid >>"))))
                assert not ids & used and max(ids) <= 15, (f, line)
                assert int(m.group(3)) * len(ids) == nthreads, line  # the groups cover the block exactly
                used |= ids
    assert groups > 0


@pytest.mark.parametrize("dtype,arith", ARITHS)
def test_adjoint_kernels_compile(dtype, arith):
    """The reverse sweep's kernels (psi and lambda in registers, gradient
    partials) compile for every parametrised gate, arithmetic and dtype."""
    before = L.lqs_jit_info()
    names = ["RX", "RY", "RZ", "PhaseShift", "Rot", "ControlledPhaseShift", "CRY", "H", "CNOT", "SWAP", "Toffoli",
             "S", "U4", "Y", "CZ"]
    c = W.random_circuit(13, 100, seed=41, names=names)
    L.lqs_jit_precompile_adjoint(13, dtype, c.ops, c.params, arith)
    after = L.lqs_jit_info()
    assert after["failed"] == before["failed"], after["last_error"]
    # a state that fits one adjoint tile compiles nothing
    c = W.ansatz(9, 2, 1)
    assert L.lqs_jit_precompile_adjoint(9, dtype, c.ops, c.params, arith) == 0


def _bank_model(src):
    """Extra shared-memory wavefronts of a generated kernel's exchanges, per
    warp and tile: each 128-byte phase of a warp access costs one wavefront
    per amplitude that shares a bank group with another lane's."""
    import re

    def swz(j, sz):
        return j ^ ((((j >> 3) ^ (j >> 6) ^ (j >> 9)) & 7) if sz == 16 else (((j >> 4) ^ (j >> 8)) & 15))

    def pfold(j, *m):
        return sum((bin(j & mb).count("1") & 1) << b for b, mb in enumerate(m))

    def obit(base, q):
        return (base >> q) & 1

    def py(expr):
        expr = re.sub(r"(0x[0-9a-f]+)u", r"\1", expr)
        expr = re.sub(r"\b(\d+)u\b", r"\1", expr)
        expr = re.sub(r"lqs::jit::swz<(\d+)>\((\w+)\)", r"swz(\2, \1)", expr)
        return expr.replace("lqs::jit::pfold", "pfold").replace("lqs::jit::obit", "obit")

    sz = 8 if "lqs::ArF32" in src else 16
    per = 128 // sz
    jt = sj = None
    named = {}
    extra = 0
    for line in src.splitlines():
        s = line.strip()
        m = re.match(r"(?:uint32_t )?jt = (.*);$", s)
        if m:
            jt = m.group(1)
        m = re.match(r"const uint32_t ((?:jo|fj)\d+) = (.*);$", s)
        if m:  # adjoint: one swizzled index for the writes of both states; fj: a folded exchange's write index
            named[m.group(1)] = (m.group(2), jt)
            continue
        m = re.match(r"\{ const uint32_t sj = (.*);$", s)
        if m:
            sj = m.group(1)
            continue
        if sj and ("st_w(&" in s or "ld_w(&" in s):
            mc = re.search(r"sj (\^|\+) (0x[0-9a-f]+)u", s)
            op, c = mc.group(1), int(mc.group(2), 16)
            for ph in range(32 // per):
                groups = {}
                for lane in range(per * ph, per * (ph + 1)):
                    env = {"swz": swz, "pfold": pfold, "obit": obit, "base": 0}
                    for nm, (ex, jt_then) in named.items():  # each under the jt of its own definition
                        env[nm] = eval(py(ex), dict(env, jt=eval(py(jt_then), {"tid": lane})))
                    env["jt"] = eval(py(jt), {"tid": lane})
                    a = eval(py(sj), env) + c if op == "+" else eval(py(sj), env) ^ c
                    groups[a % per] = groups.get(a % per, 0) + 1
                extra += max(groups.values()) - 1
        elif sj and s.startswith("}"):
            sj = None
    return extra


def _unordered_accesses(src):
    """Shared-memory accesses of a generated kernel's tile loop that conflict
    (same exchange-buffer position, different warps, at least one a write)
    without a chain of barriers ordering them.  The loop body is replayed from
    its source: exchange writes and reads with their swizzled positions per
    thread, and every barrier with the warp groups it joins (a named barrier
    joins the warps agreeing on its tid bits, __syncwarp one warp,
    __syncthreads all)."""
    import re

    def swz(j, sz):
        return j ^ ((((j >> 3) ^ (j >> 6) ^ (j >> 9)) & 7) if sz == 16 else (((j >> 4) ^ (j >> 8)) & 15))

    def pfold(j, *m):
        return sum((bin(j & mb).count("1") & 1) << b for b, mb in enumerate(m))

    def obit(base, q):
        return (base >> q) & 1

    def ev(expr, **kw):
        expr = re.sub(r"(0x[0-9a-f]+)u", r"\1", expr)
        expr = re.sub(r"(\d+)u\b", r"\1", expr)
        expr = re.sub(r"lqs::jit::swz<(\d+)>\((\w+)\)", r"swz(\2, \1)", expr).replace("lqs::jit::pfold", "pfold")
        expr = expr.replace("lqs::jit::obit", "obit")
        return eval(expr, {"swz": swz, "pfold": pfold, "obit": obit, "base": 0}, kw)

    nth = int(re.search(r"__launch_bounds__\((\d+),", src).group(1))
    nw = nth // 32
    body = re.split(r"for \(; t < G\.ntiles; t \+= [^)]*\) \{", src, maxsplit=1)[1]
    events = []  # ("bar", key(warp)) or ("acc", buf, is_write, {position: warp})
    jt = named = None
    named = {}
    sj = None
    cur = None
    for line in body.splitlines():
        s = line.strip()
        m = re.match(r"(?:uint32_t )?jt = (.*);$", s)
        if m:
            jt = [ev(m.group(1), tid=t) for t in range(nth)]
            continue
        m = re.match(r"const uint32_t ((?:jo|fj)\d+) = (.*);$", s)
        if m:
            named[m.group(1)] = [ev(m.group(2), jt=jt[t], **{k: v[t] for k, v in named.items()}) for t in range(nth)]
            continue
        m = re.match(r"\{ const uint32_t sj = (.*);$", s)
        if m:
            sj = [ev(m.group(1), jt=jt[t], **{k: v[t] for k, v in named.items()}) for t in range(nth)]
            cur = None
            continue
        m = re.search(r"(st_w|ld_w)\(&(X[ABCD])\[sj (\^|\+) (0x[0-9a-f]+)u\]", s)
        if m and sj is not None:
            wr, buf, op, c = m.group(1) == "st_w", m.group(2), m.group(3), int(m.group(4), 16)
            if cur is None or cur[1] != buf or cur[2] != wr:
                cur = ["acc", buf, wr, {}]
                events.append(cur)
            for t in range(nth):
                cur[3][sj[t] + c if op == "+" else sj[t] ^ c] = t // 32
            continue
        if s.startswith("}"):
            sj = None
            cur = None
        if "__syncthreads" in s:
            events.append(("bar", lambda w: 0))
        elif "__syncwarp" in s:
            events.append(("bar", lambda w: w))
        else:
            m = re.search(r"bar_group\((\d+)u(.*), (\d+)u\);", s)
            if m:
                bits = [int(b) for b in re.findall(r"tid >> (\d+)", m.group(2))]
                events.append(("bar", lambda w, bits=tuple(bits): tuple(((w * 32) >> b) & 1 for b in bits)))

    def ordered(v, i1, w, i2):
        seen = {v}
        for e in events[i1 + 1:i2]:
            if e[0] == "bar":
                keys = {e[1](u) for u in seen}
                seen = {x for x in range(nw) if e[1](x) in keys}
        return w in seen

    bad = []
    last = {}  # (buf, pos) -> (last write (warp, i), [reads since])
    for i, e in enumerate(events):
        if e[0] != "acc":
            continue
        _, buf, wr, own = e
        for pos, w in own.items():
            lw, rs = last.get((buf, pos), (None, []))
            deps = ([lw] if lw else []) + (rs if wr else [])
            for v, j in deps:
                if v != w and not ordered(v, j, w, i):
                    bad.append((buf, pos, v, j, w, i))
            if wr:
                last[(buf, pos)] = ((w, i), [])
            else:
                last[(buf, pos)] = (lw, rs + [(w, i)])
        if len(bad) > 20:
            break
    return bad


def test_exchanges_are_bank_conflict_free(tmp_path, monkeypatch):
    """Every layout exchange of generated kernels (forward and adjoint, both
    amplitude sizes) writes and reads shared memory without bank conflicts:
    each exchange gets a swizzle that is one-to-one on the lane positions of
    both the writing and the reading layout."""
    import glob
    monkeypatch.setenv("LQS_JIT_DUMP", str(tmp_path))
    for dtype, arith in (("c128", L.LQS_ARITH_DF), ("c64", L.LQS_ARITH_AUTO)):
        c = W.ansatz(24, 4, 3)
        L.lqs_jit_precompile(24, dtype, c.ops, c.params, arith)
        c = W.random_circuit(19, 120, seed=64)
        L.lqs_jit_precompile(19, dtype, c.ops, c.params, arith)
        L.lqs_jit_precompile_adjoint(19, dtype, c.ops, c.params, arith)
    files = glob.glob(str(tmp_path / "*.cu"))
    assert files
    bad = {f: e for f in files for e in [_bank_model(open(f).read())] if e}
    assert not bad, bad
    # and every pair of conflicting exchange accesses is ordered by barriers
    races = {f: r[:3] for f in files for r in [_unordered_accesses(open(f).read())] if r}
    assert not races, races


def test_permutation_runs_fold_into_exchanges(tmp_path, monkeypatch):
    """CNOT ladders in compiled segments are folded into the layout exchange
    that follows them (each amplitude written to its permuted position):
    generated kernels of the 30-qubit ansatz carry folded exchanges, and the
    folds stay free of bank conflicts and unordered buffer accesses."""
    import glob
    monkeypatch.setenv("LQS_JIT_DUMP", str(tmp_path))
    c = W.ansatz(30, 3, 3)
    L.lqs_jit_precompile(30, "c128", c.ops, c.params, L.LQS_ARITH_DF)
    c = W.ansatz(19, 3, 4)
    L.lqs_jit_precompile_adjoint(19, "c128", c.ops, c.params, L.LQS_ARITH_DF)
    files = glob.glob(str(tmp_path / "*.cu"))
    folded = [f for f in files if "const uint32_t fj" in open(f).read()]
    assert any("lqs_seg_" in f for f in folded) and any("lqs_adj_" in f for f in folded)
    assert any("lqs::jit::obit(base" in open(f).read() for f in folded)  # a ladder step controlled from outside
    bad = {f: e for f in folded for e in [_bank_model(open(f).read())] if e}
    assert not bad, bad
    races = {f: r[:3] for f in folded for r in [_unordered_accesses(open(f).read())] if r}
    assert not races, races
