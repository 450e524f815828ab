"""hx: matrix-free hyperelastic tangent and residual operators on GB300."""
