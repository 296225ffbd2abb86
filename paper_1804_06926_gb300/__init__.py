"""GB300-native exact triangle counting (filtered, degree-oriented set intersection)."""
