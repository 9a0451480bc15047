"""GB300-native space-variant elliptical filtering with radially-uniform box splines."""
