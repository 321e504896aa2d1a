"""Kernel descriptors on the host: validation of the declaration and a
cross-compile of the generated source for sm_103a (no GPU needed)."""
import pytest

from paper_1201_2118_gb300.descriptor import (MAX_ARRAYS, MAX_PARAMS, Descriptor,
                                              compile_source, generate)


def _uv(**kw):
    args = dict(name="update_velocity",
                inputs={"wu": "cached", "wv": "cached", "ww": "cached", "p": "cached"},
                outputs=["u", "v", "w"], params=["cdt"], stencil=(0, 1, 0, 1, 0, 1),
                body="""
                  const float pc = at(p, 0, 0, 0);
                  out(u) = at(wu, 0, 0, 0) - cdt * ((at(p, 1, 0, 0) - pc) * idx);
                  out(v) = at(wv, 0, 0, 0) - cdt * ((at(p, 0, 1, 0) - pc) * idy);
                  out(w) = at(ww, 0, 0, 0) - cdt * ((at(p, 0, 0, 1) - pc) * idz);
                """)
    args.update(kw)
    return Descriptor(**args)


def test_valid_descriptor_generates_one_kernel_and_launcher():
    src = generate(_uv())
    assert src.count("__global__") == 1
    assert 'extern "C" int gen_update_velocity_launch' in src
    assert "at(" not in src and "out(" not in src.split("gen_update_velocity(GenArgs")[1]


@pytest.mark.parametrize("body,msg", [
    ("out(u) = at(p, -1, 0, 0); out(v) = 0.f; out(w) = 0.f;", "outside the declared stencil"),
    ("out(u) = at(q, 0, 0, 0); out(v) = 0.f; out(w) = 0.f;", "not an input"),
    ("out(u) = at(p, 0, 0, 0); out(v) = 0.f;", "never assigned"),
    ("out(u) = 0.f; out(v) = 0.f; out(w) = 0.f; out(p) = 1.f;", "not an output"),
    ("out(u) = at(p, i, 0, 0); out(v) = 0.f; out(w) = 0.f;", "integer literals"),
])
def test_body_errors(body, msg):
    with pytest.raises(ValueError, match=msg):
        _uv(body=body).validate()


def test_declaration_errors():
    with pytest.raises(ValueError, match="mode"):
        _uv(inputs={"wu": "cached", "wv": "cached", "ww": "cached", "p": "maybe"}).validate()
    with pytest.raises(ValueError, match="reserved"):
        _uv(params=["idx"]).validate()
    with pytest.raises(ValueError, match="distinct"):
        _uv(params=["p"]).validate()
    with pytest.raises(ValueError, match="stencil"):
        _uv(stencil=(0, 3, 0, 1, 0, 1)).validate()
    with pytest.raises(ValueError, match="shared memory"):
        _uv(stencil=(2, 2, 2, 2, 2, 2), ty=16).validate()
    with pytest.raises(ValueError, match="identifier"):
        _uv(name="update-velocity").validate()
    with pytest.raises(ValueError, match="at least one output"):
        _uv(outputs=[], body="const float x = at(p, 0, 0, 0);").validate()
    with pytest.raises(ValueError, match="at most"):
        _uv(params=["c%d" % k for k in range(MAX_PARAMS + 1)]).validate()
    with pytest.raises(ValueError, match="at most"):
        _uv(inputs={"in%d" % k: "direct" for k in range(MAX_ARRAYS)}).validate()
    for ty, zc in ((3, 32), (32, 32), (8, 0), (8, 1025)):
        with pytest.raises(ValueError, match="ty must be"):
            _uv(ty=ty, zc=zc).validate()
    with pytest.raises(ValueError, match="stencil"):
        _uv(stencil=(0, 1, 0, 1, 0)).validate()
    # the limits themselves are accepted
    _uv(ty=16, zc=1024).validate()
    _uv(ty=1, zc=1).validate()


def test_generated_source_cross_compiles_for_sm103a():
    path = compile_source(generate(_uv()), "update_velocity")
    assert path.endswith(".so")
