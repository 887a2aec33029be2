"""The bench's work accounting, restated from the network's layer shapes and
the per-unit figures: MLP adjoint MACs per point, and the flops of a phasor
call in either form (no GPU)."""
import geraf_inputs as gi


def test_mlp_adjoint_macs_from_layer_shapes():
    import bench
    spec = gi.MLPSpec()
    shapes = spec.shapes()                       # [(out, in)] hidden layers, then the head
    streams = 4                                  # the value and three tangents
    macs = 0
    for li, (o, i) in enumerate(shapes):
        macs += streams * o * i                  # weight gradient
        if li > 0:
            macs += streams * o * i              # adjoint of the layer input (not of the encoding)
    assert macs == bench.mlp_backward_macs(spec) == 413696


def test_phasor_call_flops():
    import bench
    pairs, n_f = 1000, 128
    # Chebyshev form: 6 flops per pair per order run (T_k recurrence FMA and the
    # complex accumulation, 2 FMA), plus the fixed per-pair work: the
    # double-single range (32), the carrier phase (3), x and 2x (4), and the
    # call's amplitude or chain rule (render 15, render adjoint 30, filter 8,
    # filter adjoint 6)
    common = 32 + 3 + 4
    assert bench.call_flops("render", pairs, n_f, 19.5) == pairs * (19.5 * 6 + common + 15)
    assert bench.call_flops("render_backward", pairs, n_f, 21.5) == pairs * (21.5 * 6 + common + 30)
    assert bench.call_flops("filter", pairs, n_f, 16.0) == pairs * (16.0 * 6 + common + 8)
    assert bench.call_flops("filter_backward", pairs, n_f, 17.0) == pairs * (17.0 * 6 + common + 6)
    # per-bin recurrence: 10 flops per term for the to-bins sums (amplitude times
    # the unit phasor, 2 FMA, and the angle-addition step, 2 MUL + 2 FMA), 8 for
    # the to-points sums (complex coefficients by Horner's rule, 4 FMA)
    assert bench.call_flops("render", pairs, n_f, 0) == pairs * n_f * 10
    assert bench.call_flops("filter_backward", pairs, n_f, 0) == pairs * n_f * 10
    assert bench.call_flops("filter", pairs, n_f, 0) == pairs * n_f * 8
    assert bench.call_flops("render_backward", pairs, n_f, 0) == pairs * n_f * 8
    assert bench.call_flops("fields_backward", 0, 0, 0, mlp_macs=413696, n_mlp_pts=10) == 2 * 413696 * 10
