"""GB300-native null-geodesic ray tracer (Kerr / Manko-Novikov, RK4, persistent ray queue)."""
